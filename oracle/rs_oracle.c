/*
 * rs_oracle.c -- plain FP64 CPU reference for the speedup-prediction / recommendation path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library.  The CUDA library shares no code with it.
 *
 * What it computes, step by step, in the paper's order:
 *   Sec. 2   feature vectors: counters normalised by the cycle count; here followed by a
 *            log transform and a per-program z-score (the reading stated below);
 *   Sec. 3.3 the 64 versions of a program are the 6-bit optimization masks; optimization j
 *            pairs a version v without j with the version v|j that adds it;
 *   Sec. 2   Tier 2 trains one model per optimization from before/after pairs: the
 *            feature vector of the "before" version, labelled with the log speedup
 *            log t(before) - log t(after);
 *   Sec. 3.4 the regression family: ridge regression with an unpenalised intercept,
 *            solved from the primal normal equations with a textbook Cholesky; or
 *   Sec. 3.4 the instance-based learner IBK: the k = 10 training instances nearest to the
 *            test vector by Euclidean distance, their labels combined into the prediction;
 *   Sec. 3.4 the M5P model tree (rs_m5p.c), for the transfer protocol;
 *   Sec. 5   evaluation: test versions are those outside the split's training set; each
 *            gets one predicted speedup per optimization it does not already contain;
 *   Sec. 2   Tier 3 sorts by expected benefit, keeps those at or above a threshold and
 *            reports at most k;
 *   Sec. 5/6 scoring: actual vs expected speedup (AC/EX) and sign accuracy (Table 3);
 *   Sec. 5   Table 2 transfer: a model trained on one set of feature vectors (one program,
 *            input and run) predicts for another set (another run, input or program).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - log(max(x / cycles, eps)) with eps = 1e-30, then population mean / standard
 *     deviation per program and feature over all its versions; sigma < 1e-12 gives z = 0;
 *   - a training pair needs both endpoints in the training set;
 *   - ridge: minimise sum (y - b - z.beta)^2 + lambda |beta|^2, lambda not scaled by n;
 *   - candidates are the optimizations not yet in the test version (a flag ranks all 6);
 *   - ties in predicted speedup rank the lower optimization index first;
 *   - the threshold is compared in log space, inclusive (pred >= log tau);
 *   - "gain" means log speedup > 0 for both predicted and actual values;
 *   - IBK: distances between z-scored feature vectors; the "mode" of the neighbours'
 *     labels, which are continuous log speedups, is read as their mean (summed in pair
 *     order); equal distances take the lower pair index first; fewer than k training
 *     pairs use all of them;
 *   - M5P: the readings listed in rs_m5p.c;
 *   - transfer (Table 2): the training set is a group of runs (one program and input, or
 *     several runs of it); their vectors are standardized together and the test set with the
 *     same statistics; a model is trained from all pairs of all runs, a pair never spanning
 *     two runs; every version of the test set is a test row, scored against the test set's
 *     own times; an optimization mask limits the candidates (the optimizations two programs
 *     share, for cross-program transfer).
 *
 * All arithmetic is double precision, in plain loops, with no blocking or reordering
 * beyond the definitions above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NOPT 6
#define ORC_FIT_OK 0
#define ORC_FIT_EMPTY 1
#define ORC_FIT_NOTPD 2
#define ORC_FIT_NONFINITE 3
#define ORC_RANK_ALL 1
#define ORC_MODEL_IBK 4
#define ORC_MODEL_M5P 8

/* The M5P model tree (rs_m5p.c). */
typedef struct orc_m5_tree orc_m5_tree_t;
int orc_m5p_tree_bytes(void);
int orc_m5p_fit_tree(int n, int F, const double* Zrows, const double* y, void* T);
double orc_m5p_predict_tree(const void* T, const double* z);
#define ORC_NCOUNTERS 16

/* ---------------------------------------------------------------------------------- */
/* Sec. 2: counter normalisation by cycles, then log and per-program z-score.         */
/* X: [V][F] raw counters (double), cycles: [V] or NULL. Outputs Z [V][F], mu, sigma. */
void orc_standardize(int V, int F, const double* X, const double* cycles, double eps,
                     double* Z, double* mu, double* sigma) {
    for (int f = 0; f < F; ++f) {
        double s = 0.0;
        for (int r = 0; r < V; ++r) {
            double x = X[(size_t)r * F + f];
            if (cycles) x = x / cycles[r];
            double l = log(x > eps ? x : eps);
            Z[(size_t)r * F + f] = l;            /* Z holds the log values for now */
            s += l;
        }
        double m = s / V;
        double q = 0.0;
        for (int r = 0; r < V; ++r) {
            double d = Z[(size_t)r * F + f] - m;
            q += d * d;
        }
        double sd = sqrt(q / V);
        for (int r = 0; r < V; ++r) {
            double l = Z[(size_t)r * F + f];
            Z[(size_t)r * F + f] = (sd > 1e-12) ? (l - m) / sd : 0.0;
        }
        mu[f] = m;
        sigma[f] = sd;
    }
}

/* ---------------------------------------------------------------------------------- */
/* Sec. 3.3: optimization j pairs version v (bit j clear) with the version whose mask is
 * m_v | (1 << j).  Brute force over all version pairs.  Returns the number of pairs.    */
int orc_pairs(int V, const uint8_t* masks, int j, int* before, int* after) {
    int n = 0;
    for (int v = 0; v < V; ++v) {
        if ((masks[v] >> j) & 1) continue;
        int target = masks[v] | (1 << j);
        for (int w = 0; w < V; ++w) {
            if (masks[w] == target) {
                before[n] = v;
                after[n] = w;
                ++n;
                break;
            }
        }
    }
    return n;
}

/* ---------------------------------------------------------------------------------- */
/* Textbook Cholesky A = L L^T of an n x n SPD matrix (row-major, lower triangle used).
 * Returns 0 on success, 1 if a pivot is not positive.  L overwrites the lower triangle. */
int orc_cholesky(int n, double* A) {
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0)) return 1;
        double ljj = sqrt(d);
        A[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = s / ljj;
        }
    }
    return 0;
}

/* Solve L L^T x = b in place (b becomes x), L from orc_cholesky. */
void orc_cholesky_solve(int n, const double* L, double* b) {
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * b[k];
        b[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * b[k];
        b[i] = s / L[(size_t)i * n + i];
    }
}

/* ---------------------------------------------------------------------------------- */
/* Sec. 3.4 regression family, read as ridge with an unpenalised intercept:
 *   minimise sum_i (y_i - b - z_i . beta)^2 + lambda * |beta|^2.
 * Plain definition: centre Z and y on the training rows, form the primal normal equations
 * (Zc^T Zc + lambda I) beta = Zc^T yc, solve by Cholesky, b = ybar - zbar . beta.
 * Zrows: [n][F].  Returns a fit status.  work needs F*F + 2*F doubles.                 */
int orc_ridge_fit(int n, int F, const double* Zrows, const double* y, double lambda,
                  double* beta, double* b, double* work) {
    if (n <= 0) {
        for (int f = 0; f < F; ++f) beta[f] = 0.0;
        *b = 0.0;
        return ORC_FIT_EMPTY;
    }
    double* G = work;
    double* zbar = work + (size_t)F * F;
    double* r = zbar + F;
    double ybar = 0.0;
    for (int i = 0; i < n; ++i) ybar += y[i];
    ybar /= n;
    for (int f = 0; f < F; ++f) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += Zrows[(size_t)i * F + f];
        zbar[f] = s / n;
    }
    for (int f = 0; f < F; ++f) {
        for (int g = 0; g <= f; ++g) {
            double s = 0.0;
            for (int i = 0; i < n; ++i)
                s += (Zrows[(size_t)i * F + f] - zbar[f]) * (Zrows[(size_t)i * F + g] - zbar[g]);
            G[(size_t)f * F + g] = s;
            G[(size_t)g * F + f] = s;
        }
        G[(size_t)f * F + f] += lambda;
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += (Zrows[(size_t)i * F + f] - zbar[f]) * (y[i] - ybar);
        r[f] = s;
    }
    if (orc_cholesky(F, G)) {
        for (int f = 0; f < F; ++f) beta[f] = 0.0;
        *b = 0.0;
        return ORC_FIT_NOTPD;
    }
    orc_cholesky_solve(F, G, r);
    double bb = ybar;
    int finite = isfinite(ybar);
    for (int f = 0; f < F; ++f) {
        beta[f] = r[f];
        bb -= zbar[f] * r[f];
        finite = finite && isfinite(r[f]);
    }
    *b = bb;
    if (!finite || !isfinite(bb)) return ORC_FIT_NONFINITE;
    return ORC_FIT_OK;
}

/* ---------------------------------------------------------------------------------- */
/* Sec. 2 Tier 3: order candidate optimizations by predicted log speedup (descending;
 * equal values keep the lower index first), keep those >= log_tau, report at most k.
 * pred[6] with valid[6] flags.  Writes the chosen indices into idx; returns the count. */
/* Sec. 3.4, IBK: the prediction for test vector zt from n training rows Zrows [n][F] with
 * labels y: squared Euclidean distances d_a = sum_f (zt_f - z_a,f)^2, the kn nearest
 * (insertion into a list ordered by (d, a), so equal distances keep the lower index first),
 * and the mean of their labels, summed in ascending index a.  Any n >= 1 (the transfer
 * protocol pools up to 32 pairs per run); 1 <= kn <= ORC_IBK_MAXK, else NaN.         */
#define ORC_IBK_MAXK 64
double orc_ibk_predict(int n, int F, const double* Zrows, const double* y, const double* zt, int kn) {
    int sel[ORC_IBK_MAXK];
    double sd[ORC_IBK_MAXK];
    int m = 0;
    if (n < 1 || kn < 1 || kn > ORC_IBK_MAXK) return NAN;
    for (int a = 0; a < n; ++a) {
        double d = 0.0;
        for (int f = 0; f < F; ++f) {
            double e = zt[f] - Zrows[(size_t)a * F + f];
            d += e * e;
        }
        /* insert (d, a) after every kept entry with distance <= d */
        int pos = m;
        while (pos > 0 && sd[pos - 1] > d) --pos;
        if (pos >= kn) continue;
        int last = m < kn ? m : kn - 1;
        for (int q = last; q > pos; --q) {
            sd[q] = sd[q - 1];
            sel[q] = sel[q - 1];
        }
        sd[pos] = d;
        sel[pos] = a;
        if (m < kn) ++m;
    }
    /* the chosen indices in ascending order (insertion sort of the m <= kn entries) */
    for (int q = 1; q < m; ++q) {
        const int cur = sel[q];
        int p = q - 1;
        while (p >= 0 && sel[p] > cur) {
            sel[p + 1] = sel[p];
            --p;
        }
        sel[p + 1] = cur;
    }
    double sum = 0.0;
    for (int q = 0; q < m; ++q) sum += y[sel[q]];
    return sum / m;
}

int orc_rank(const double* pred, const int* valid, int k, double log_tau, int* idx) {
    int order[ORC_NOPT];
    int m = 0;
    for (int j = 0; j < ORC_NOPT; ++j)
        if (valid[j]) order[m++] = j;
    /* insertion sort: a later element moves ahead only if strictly larger */
    for (int a = 1; a < m; ++a) {
        int cur = order[a];
        int b = a - 1;
        while (b >= 0 && pred[order[b]] < pred[cur]) {
            order[b + 1] = order[b];
            --b;
        }
        order[b + 1] = cur;
    }
    int c = 0;
    for (int a = 0; a < m && c < k; ++a) {
        if (pred[order[a]] >= log_tau) idx[c++] = order[a];
    }
    return c;
}

static int popcount64(uint64_t x) {
    int c = 0;
    while (x) {
        x &= x - 1;
        ++c;
    }
    return c;
}

/* ---------------------------------------------------------------------------------- */
/* Number of test rows (versions outside the training set) of each split, and their
 * exclusive prefix sum: rec_offsets[S+1].                                             */
void orc_rec_offsets(int P, const int64_t* row_offsets, const int64_t* split_offsets,
                     const uint64_t* train_masks, int64_t* rec_offsets) {
    int64_t acc = 0;
    for (int p = 0; p < P; ++p) {
        int V = (int)(row_offsets[p + 1] - row_offsets[p]);
        uint64_t full = (V >= 64) ? ~0ull : ((1ull << V) - 1ull);
        for (int64_t s = split_offsets[p]; s < split_offsets[p + 1]; ++s) {
            rec_offsets[s] = acc;
            acc += V - popcount64(train_masks[s] & full);
        }
    }
    rec_offsets[split_offsets[P]] = acc;
}

/* ---------------------------------------------------------------------------------- */
/* Whole cross-validation pass over a batch of programs (Sec. 5's protocol, with the
 * train/test split given as a bit mask over each program's versions).
 *
 * Inputs: P programs; program p owns rows row_offsets[p]..row_offsets[p+1]-1 of masks,
 * log_time and cycles, and a row-major [V_p][F_p] block of X at element x_offsets[p]
 * (X double, or float when x_is_f32).  Splits split_offsets[p]..split_offsets[p+1]-1
 * belong to program p.
 * Outputs (any may be NULL except counters): Z [same layout as X, double], mu/sigma
 * [same offsets as one row per program: x_offsets scaled, see below], fit_status [S][6],
 * rec_code [R] (bits 0-3 count, then 4 bits per recommended optimization, unused 0xF),
 * rec_pred [R][k], pred_all [R][6] (NaN where no prediction), counters [16] (added to).
 * mu/sigma are indexed by feat_offsets[p] + f (feat_offsets = prefix sum of F_p).
 * rec rows are ordered by split, then by version slot.                                */
void orc_cv_batch(int P, const int64_t* row_offsets, const int32_t* feat_width,
                  const int64_t* x_offsets, const int64_t* feat_offsets, const void* Xv,
                  int x_is_f32, const uint8_t* masks, const double* log_time,
                  const double* cycles, const int64_t* split_offsets,
                  const uint64_t* train_masks, double lambda, int k, double log_tau,
                  int flags, double eps, double* Z_out, double* mu_out, double* sigma_out,
                  uint8_t* fit_status, const int64_t* rec_offsets, uint32_t* rec_code,
                  double* rec_pred, double* pred_all, uint64_t* counters, int nthreads, int ibk_k) {
    (void)nthreads;
    int64_t S = split_offsets[P];
    uint64_t* per_split = (uint64_t*)calloc((size_t)(S > 0 ? S : 1) * ORC_NCOUNTERS, sizeof(uint64_t));
    for (int p = 0; p < P; ++p) {
        int V = (int)(row_offsets[p + 1] - row_offsets[p]);
        int F = feat_width[p];
        int64_t r0 = row_offsets[p];
        double* X = (double*)malloc(sizeof(double) * (size_t)V * F);
        double* Z = (double*)malloc(sizeof(double) * (size_t)V * F);
        double* mu = (double*)malloc(sizeof(double) * F);
        double* sg = (double*)malloc(sizeof(double) * F);
        for (int64_t e = 0; e < (int64_t)V * F; ++e)
            X[e] = x_is_f32 ? (double)((const float*)Xv)[x_offsets[p] + e]
                            : ((const double*)Xv)[x_offsets[p] + e];
        orc_standardize(V, F, X, cycles ? cycles + r0 : NULL, eps, Z, mu, sg);
        if (Z_out) memcpy(Z_out + x_offsets[p], Z, sizeof(double) * (size_t)V * F);
        if (mu_out) memcpy(mu_out + feat_offsets[p], mu, sizeof(double) * F);
        if (sigma_out) memcpy(sigma_out + feat_offsets[p], sg, sizeof(double) * F);
        const uint8_t* pm = masks + r0;
        const double* lt = log_time + r0;

        /* all pairs of the program, per optimization (Sec. 3.3) */
        int pb[ORC_NOPT][64], pa[ORC_NOPT][64], np_[ORC_NOPT];
        for (int j = 0; j < ORC_NOPT; ++j) np_[j] = orc_pairs(V, pm, j, pb[j], pa[j]);
        /* slot of each mask in this program, -1 if absent (for actual speedups) */
        int slot_of[64];
        for (int m = 0; m < 64; ++m) slot_of[m] = -1;
        for (int v = 0; v < V; ++v) slot_of[pm[v]] = v;
        uint64_t full = (V >= 64) ? ~0ull : ((1ull << V) - 1ull);

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
        for (int64_t s = split_offsets[p]; s < split_offsets[p + 1]; ++s) {
            uint64_t T = train_masks[s] & full;
            uint64_t* cnt = per_split + (size_t)s * ORC_NCOUNTERS;
            double* beta = (double*)malloc(sizeof(double) * ORC_NOPT * F);
            double bias[ORC_NOPT];
            int ok[ORC_NOPT];
            double* work = (double*)malloc(sizeof(double) * ((size_t)F * F + 2 * (size_t)F));
            /* the training pairs of each optimization: before-version rows and labels */
            double* Zr = (double*)malloc(sizeof(double) * ORC_NOPT * 64 * (size_t)F);
            double yv[ORC_NOPT][64];
            int nj[ORC_NOPT];
            const int ibk = (flags & ORC_MODEL_IBK) != 0;
            for (int j = 0; j < ORC_NOPT; ++j) {
                int n = 0;
                double* Zj = Zr + (size_t)j * 64 * F;
                for (int q = 0; q < np_[j]; ++q) {
                    int v = pb[j][q], w = pa[j][q];
                    if (((T >> v) & 1) && ((T >> w) & 1)) {
                        memcpy(Zj + (size_t)n * F, Z + (size_t)v * F, sizeof(double) * F);
                        yv[j][n] = lt[v] - lt[w];   /* log speedup of adding j (Sec. 5) */
                        ++n;
                    }
                }
                nj[j] = n;
                int st;
                if (ibk)   /* IBK stores the instances; a model exists when there is one */
                    st = n > 0 ? ORC_FIT_OK : ORC_FIT_EMPTY;
                else
                    st = orc_ridge_fit(n, F, Zj, yv[j], lambda, beta + (size_t)j * F, &bias[j], work);
                ok[j] = (st == ORC_FIT_OK);
                if (fit_status) fit_status[s * ORC_NOPT + j] = (uint8_t)st;
                cnt[9 + st] += 1;
            }
            int64_t row = rec_offsets[s];
            for (int t = 0; t < V; ++t) {
                if ((T >> t) & 1) continue;
                double pred[ORC_NOPT], act[ORC_NOPT];
                int valid[ORC_NOPT], known[ORC_NOPT];
                for (int j = 0; j < ORC_NOPT; ++j) {
                    int cand = (flags & ORC_RANK_ALL) || !((pm[t] >> j) & 1);
                    valid[j] = 0;
                    known[j] = 0;
                    pred[j] = NAN;
                    act[j] = NAN;
                    if (!cand) continue;
                    if (!ok[j]) {
                        cnt[13] += 1;
                        continue;
                    }
                    double yh;
                    if (ibk) {
                        yh = orc_ibk_predict(nj[j], F, Zr + (size_t)j * 64 * F, yv[j], Z + (size_t)t * F, ibk_k);
                    } else {
                        yh = bias[j];
                        for (int f = 0; f < F; ++f) yh += Z[(size_t)t * F + f] * beta[(size_t)j * F + f];
                    }
                    pred[j] = yh;
                    valid[j] = 1;
                    cnt[1] += 1;
                    if (!((pm[t] >> j) & 1)) {
                        int w = slot_of[pm[t] | (1 << j)];
                        if (w >= 0) {
                            act[j] = lt[t] - lt[w];
                            known[j] = 1;
                        }
                    }
                    if (known[j]) {
                        cnt[2] += 1;
                        if ((pred[j] > 0.0) == (act[j] > 0.0)) cnt[3] += 1;
                    }
                }
                int idx[ORC_NOPT];
                int c = orc_rank(pred, valid, k, log_tau, idx);
                uint32_t code = (uint32_t)c;
                for (int a = 0; a < ORC_NOPT; ++a)
                    code |= (uint32_t)(a < c ? idx[a] : 0xF) << (4 + 4 * a);
                if (rec_code) rec_code[row] = code;
                if (rec_pred)
                    for (int a = 0; a < k; ++a) rec_pred[row * k + a] = a < c ? pred[idx[a]] : NAN;
                if (pred_all)
                    for (int j = 0; j < ORC_NOPT; ++j) pred_all[row * ORC_NOPT + j] = pred[j];
                cnt[0] += 1;
                cnt[4] += (uint64_t)c;
                for (int a = 0; a < c; ++a) {
                    if (known[idx[a]]) {
                        cnt[5] += 1;
                        if (act[idx[a]] > 0.0) cnt[6] += 1;
                    }
                }
                /* top-1 agreement over the scored candidates of this row */
                int bp = -1, ba = -1;
                for (int j = 0; j < ORC_NOPT; ++j) {
                    if (!(valid[j] && known[j])) continue;
                    if (bp < 0 || pred[j] > pred[bp]) bp = j;
                    if (ba < 0 || act[j] > act[ba]) ba = j;
                }
                if (bp >= 0) {
                    cnt[7] += 1;
                    if (bp == ba) cnt[8] += 1;
                }
                ++row;
            }
            free(beta);
            free(work);
            free(Zr);
        }
        free(X);
        free(Z);
        free(mu);
        free(sg);
    }
    for (int64_t s = 0; s < S; ++s)
        for (int c = 0; c < ORC_NCOUNTERS; ++c) counters[c] += per_split[(size_t)s * ORC_NCOUNTERS + c];
    free(per_split);
}

/* Sec. 5, Table 2: train on a group of runs of set A, predict and score a program of set B.
 * Problem q trains on runs group_offsets[q] .. group_offsets[q+1]-1 of A (each run laid out
 * like one program of orc_cv_batch's input: a_row_offsets, a_feat_width, a_x_offsets, a_X,
 * a_masks, a_log_time, a_cycles) and tests on program q of B (b_row_offsets, b_x_offsets,
 * b_X, b_masks, b_log_time, b_cycles), which has the runs' feature width.  For each q: the
 * vectors of all the group's runs are standardized together (mu, sigma over all of them),
 * B's program with those statistics; per optimization j the training pairs are the
 * before/after pairs of every run (Sec. 3.3; a pair never spans two runs), run by run, in
 * ascending before slot, labelled with that run's log speedups; the model (ridge, or IBK
 * with ORC_MODEL_IBK) predicts for every version t of B's program its candidates j (not in
 * t's mask, or all six with ORC_RANK_ALL) that are also in opt_mask; ranking, threshold and
 * scoring as in orc_cv_batch with B's times for the actual speedups.  Test rows: B's
 * versions, program by program, in slot order (R = B's row total).  fit_status [Q][6].     */
void orc_transfer(int Q, const int64_t* group_offsets, const int32_t* a_feat_width,
                  const int64_t* a_row_offsets, const int64_t* a_x_offsets, const double* a_X,
                  const uint8_t* a_masks, const double* a_log_time, const double* a_cycles,
                  const int64_t* b_row_offsets, const int64_t* b_x_offsets, const double* b_X,
                  const uint8_t* b_masks, const double* b_log_time, const double* b_cycles,
                  double lambda, int k, double log_tau, int flags, int opt_mask, int ibk_k, double eps,
                  uint8_t* fit_status, uint32_t* rec_code, double* rec_pred, double* pred_all,
                  uint64_t* counters) {
    const int ibk = (flags & ORC_MODEL_IBK) != 0;
    const int m5p = !ibk && (flags & ORC_MODEL_M5P) != 0;
    void* trees = m5p ? malloc((size_t)orc_m5p_tree_bytes() * ORC_NOPT) : NULL;
    int64_t row = 0;
    for (int q = 0; q < Q; ++q) {
        const int64_t g0 = group_offsets[q], g1 = group_offsets[q + 1];
        const int F = a_feat_width[g0];
        int N = 0;                                   /* versions of all runs of the group */
        for (int64_t r = g0; r < g1; ++r) N += (int)(a_row_offsets[r + 1] - a_row_offsets[r]);
        const int VB = (int)(b_row_offsets[q + 1] - b_row_offsets[q]);
        const int64_t rb = b_row_offsets[q];
        double* XA = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * F);
        double* CA = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        double* LA = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        double* ZA = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * F);
        double* ZB = (double*)malloc(sizeof(double) * (size_t)(VB > 0 ? VB : 1) * F);
        double* mu = (double*)malloc(sizeof(double) * F);
        double* sg = (double*)malloc(sizeof(double) * F);
        int u = 0;
        for (int64_t r = g0; r < g1; ++r) {          /* the runs' rows, one after another */
            const int V = (int)(a_row_offsets[r + 1] - a_row_offsets[r]);
            for (int v = 0; v < V; ++v, ++u) {
                memcpy(XA + (size_t)u * F, a_X + a_x_offsets[r] + (int64_t)v * F, sizeof(double) * F);
                CA[u] = a_cycles ? a_cycles[a_row_offsets[r] + v] : 1.0;
                LA[u] = a_log_time[a_row_offsets[r] + v];
            }
        }
        orc_standardize(N, F, XA, a_cycles ? CA : NULL, eps, ZA, mu, sg);
        for (int t = 0; t < VB; ++t)        /* B with A's statistics */
            for (int f = 0; f < F; ++f) {
                double x = b_X[b_x_offsets[q] + (int64_t)t * F + f];
                if (b_cycles) x = x / b_cycles[rb + t];
                double l = log(x > eps ? x : eps);
                ZB[(size_t)t * F + f] = (sg[f] > 1e-12) ? (l - mu[f]) / sg[f] : 0.0;
            }
        const uint8_t* mb = b_masks + rb;
        const double* ltb = b_log_time + rb;
        const size_t cap = (size_t)(N > 0 ? N : 1);  /* pairs per optimization <= versions */
        double* beta = (double*)malloc(sizeof(double) * ORC_NOPT * F);
        double* work = (double*)malloc(sizeof(double) * ((size_t)F * F + 2 * (size_t)F));
        double* Zr = (double*)malloc(sizeof(double) * ORC_NOPT * cap * F);
        double* yv = (double*)malloc(sizeof(double) * ORC_NOPT * cap);
        double bias[ORC_NOPT];
        int nj[ORC_NOPT], ok[ORC_NOPT];
        for (int j = 0; j < ORC_NOPT; ++j) {
            double* Zj = Zr + (size_t)j * cap * F;
            double* yj = yv + (size_t)j * cap;
            int n = 0, u0 = 0;
            for (int64_t r = g0; r < g1; ++r) {      /* pairs within each run (Sec. 3.3) */
                const int V = (int)(a_row_offsets[r + 1] - a_row_offsets[r]);
                int before[64], after[64];
                const int np = orc_pairs(V, a_masks + a_row_offsets[r], j, before, after);
                for (int e = 0; e < np; ++e, ++n) {
                    memcpy(Zj + (size_t)n * F, ZA + (size_t)(u0 + before[e]) * F, sizeof(double) * F);
                    yj[n] = LA[u0 + before[e]] - LA[u0 + after[e]];
                }
                u0 += V;
            }
            nj[j] = n;
            int st;
            if (ibk) st = n > 0 ? ORC_FIT_OK : ORC_FIT_EMPTY;
            else if (m5p)
                st = n == 0 ? ORC_FIT_EMPTY
                            : (orc_m5p_fit_tree(n, F, Zj, yj, (char*)trees + (size_t)j * orc_m5p_tree_bytes())
                                   ? ORC_FIT_NOTPD : ORC_FIT_OK);
            else st = orc_ridge_fit(n, F, Zj, yj, lambda, beta + (size_t)j * F, &bias[j], work);
            ok[j] = st == ORC_FIT_OK;
            if (fit_status) fit_status[q * ORC_NOPT + j] = (uint8_t)st;
            counters[9 + st] += 1;
        }
        int slot_of[64];
        for (int m = 0; m < 64; ++m) slot_of[m] = -1;
        for (int v = 0; v < VB; ++v) slot_of[mb[v]] = v;
        for (int t = 0; t < VB; ++t, ++row) {
            double pred[ORC_NOPT], act[ORC_NOPT];
            int valid[ORC_NOPT], known[ORC_NOPT];
            for (int j = 0; j < ORC_NOPT; ++j) {
                const int cand = ((flags & ORC_RANK_ALL) || !((mb[t] >> j) & 1)) && ((opt_mask >> j) & 1);
                valid[j] = known[j] = 0;
                pred[j] = act[j] = NAN;
                if (!cand) continue;
                if (!ok[j]) {
                    counters[13] += 1;
                    continue;
                }
                double yh;
                if (ibk) {
                    yh = orc_ibk_predict(nj[j], F, Zr + (size_t)j * cap * F, yv + (size_t)j * cap,
                                         ZB + (size_t)t * F, ibk_k);
                } else if (m5p) {
                    yh = orc_m5p_predict_tree((char*)trees + (size_t)j * orc_m5p_tree_bytes(), ZB + (size_t)t * F);
                } else {
                    yh = bias[j];
                    for (int f = 0; f < F; ++f) yh += ZB[(size_t)t * F + f] * beta[(size_t)j * F + f];
                }
                pred[j] = yh;
                valid[j] = 1;
                counters[1] += 1;
                if (!((mb[t] >> j) & 1)) {
                    const int w = slot_of[mb[t] | (1 << j)];
                    if (w >= 0) {
                        act[j] = ltb[t] - ltb[w];
                        known[j] = 1;
                    }
                }
                if (known[j]) {
                    counters[2] += 1;
                    if ((pred[j] > 0.0) == (act[j] > 0.0)) counters[3] += 1;
                }
            }
            int idx[ORC_NOPT];
            const int c = orc_rank(pred, valid, k, log_tau, idx);
            uint32_t code = (uint32_t)c;
            for (int a = 0; a < ORC_NOPT; ++a) code |= (uint32_t)(a < c ? idx[a] : 0xF) << (4 + 4 * a);
            if (rec_code) rec_code[row] = code;
            if (rec_pred)
                for (int a = 0; a < k; ++a) rec_pred[row * k + a] = a < c ? pred[idx[a]] : NAN;
            if (pred_all)
                for (int j = 0; j < ORC_NOPT; ++j) pred_all[row * ORC_NOPT + j] = pred[j];
            counters[0] += 1;
            counters[4] += (uint64_t)c;
            for (int a = 0; a < c; ++a)
                if (known[idx[a]]) {
                    counters[5] += 1;
                    if (act[idx[a]] > 0.0) counters[6] += 1;
                }
            int bp = -1, ba = -1;
            for (int j = 0; j < ORC_NOPT; ++j) {
                if (!(valid[j] && known[j])) continue;
                if (bp < 0 || pred[j] > pred[bp]) bp = j;
                if (ba < 0 || act[j] > act[ba]) ba = j;
            }
            if (bp >= 0) {
                counters[7] += 1;
                if (bp == ba) counters[8] += 1;
            }
        }
        free(XA);
        free(CA);
        free(LA);
        free(ZA);
        free(ZB);
        free(mu);
        free(sg);
        free(beta);
        free(work);
        free(Zr);
        free(yv);
    }
    free(trees);
}

int orc_num_threads_available(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
