/*
 * rs_m5p.c -- plain FP64 CPU reference of the M5P model tree (TEST INFRASTRUCTURE ONLY).
 *
 * Sec. 3.4 names M5P (a model tree) beside IBK; the paper gives no algorithm, so this follows
 * the published description of M5' (Wang and Witten 1997, after Quinlan's M5, 1992):
 *
 *   grow    a node with fewer than 4 instances, or whose label standard deviation is at most
 *           5 % of the root's, is a leaf; otherwise it is split on the attribute and threshold
 *           that maximise the standard deviation reduction
 *               SDR = sd(S) - (|L| sd(L) + |R| sd(R)) / |S|
 *           over thresholds halfway between consecutive distinct values of an attribute, with
 *           at least 2 instances on each side (ties: lower attribute, then lower threshold);
 *           no split with SDR > 0 makes a leaf; instances with z <= threshold go left;
 *   models  every node gets a linear model (least squares with an intercept) on the
 *           attributes tested in splits of its subtree -- as pruned so far, since the
 *           children are modelled and pruned first -- simplified by greedy elimination:
 *           while dropping one attribute (the one giving the lowest estimate) does not raise
 *           the estimated error, drop it; estimated error = mean |residual| on the node's
 *           instances x (m + v) / (m - v), m instances, v = terms + 1 (infinite if m <= v);
 *   prune   bottom-up, a subtree is replaced by its node's model when the model's estimated
 *           error is at most the subtree's (the children's errors weighted by instances);
 *   smooth  a prediction starts at the leaf's model and is blended with each ancestor's
 *           model on the way up: p = (n_c p + k q) / (n_c + k), n_c the instances of the
 *           child on the path, q the ancestor's model at the same vector, k = 15.
 *
 * Readings (the description leaves them open): sd(S) = sqrt(max(0, (s2 - s1 * s1 / c) / c)) with
 * c, s1, s2 the count, sum and sum of squares of the labels, accumulated in the order of the
 * instances (for split candidates: sorted by the attribute, ties by instance index); linear
 * models solve (G + 1e-8 I) w = r with G, r the centred normal equations (sums in instance
 * order) by the textbook Cholesky of rs_oracle.c, the 1e-8 only guarding exactly collinear
 * attributes; attributes of a model in ascending order.  All arithmetic is FP64 with no
 * contraction, in the loop orders written here.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define M5_MIN_SPLIT 4
#define M5_MIN_SIDE 2
#define M5_SD_FRAC 0.05
#define M5_SMOOTH_K 15.0
#define M5_LM_RIDGE 1e-8
#define M5_MAX_N 128
#define M5_MAX_NODES (2 * M5_MAX_N)
#define M5_MAX_TERMS 64

int orc_cholesky(int n, double* A);
void orc_cholesky_solve(int n, const double* L, double* b);

typedef struct {
    int n_nodes;
    int attr[M5_MAX_NODES];          /* split attribute, -1 for a leaf */
    double thr[M5_MAX_NODES];
    int left[M5_MAX_NODES], right[M5_MAX_NODES], parent[M5_MAX_NODES];
    int count[M5_MAX_NODES];         /* training instances reaching the node */
    int nterm[M5_MAX_NODES];
    int term_attr[M5_MAX_NODES][M5_MAX_TERMS];
    double term_w[M5_MAX_NODES][M5_MAX_TERMS];
    double b[M5_MAX_NODES];
    double est[M5_MAX_NODES];        /* estimated error after pruning */
} orc_m5_tree;

static double m5_sd(int c, double s1, double s2) {
    double v = (s2 - s1 * s1 / c) / c;
    return sqrt(v > 0.0 ? v : 0.0);
}

/* instance indices of a node, ascending */
typedef struct {
    int m;
    int idx[M5_MAX_N];
} m5_set;

/* A linear model on attributes `as` (na of them, ascending) fitted to the instances of S:
 * centred normal equations, Cholesky, intercept; writes w and b, returns the estimated
 * error (DBL_MAX when m <= na + 1 or the system fails). */
static double m5_fit_lm(const m5_set* S, int F, const double* Z, const double* y, const int* as, int na,
                        double* w, double* bout) {
    const int m = S->m;
    double ybar = 0.0;
    for (int a = 0; a < m; ++a) ybar += y[S->idx[a]];
    ybar /= m;
    double zbar[M5_MAX_TERMS];
    for (int f = 0; f < na; ++f) {
        double s = 0.0;
        for (int a = 0; a < m; ++a) s += Z[(size_t)S->idx[a] * F + as[f]];
        zbar[f] = s / m;
    }
    double G[M5_MAX_TERMS * M5_MAX_TERMS], r[M5_MAX_TERMS];
    for (int f = 0; f < na; ++f) {
        for (int g = 0; g <= f; ++g) {
            double s = 0.0;
            for (int a = 0; a < m; ++a) {
                const double* z = Z + (size_t)S->idx[a] * F;
                s += (z[as[f]] - zbar[f]) * (z[as[g]] - zbar[g]);
            }
            G[f * na + g] = s;
            G[g * na + f] = s;
        }
        G[f * na + f] += M5_LM_RIDGE;
        double s = 0.0;
        for (int a = 0; a < m; ++a) s += (Z[(size_t)S->idx[a] * F + as[f]] - zbar[f]) * (y[S->idx[a]] - ybar);
        r[f] = s;
    }
    if (na > 0) {
        if (orc_cholesky(na, G)) return DBL_MAX;
        orc_cholesky_solve(na, G, r);
    }
    double b = ybar;
    for (int f = 0; f < na; ++f) {
        w[f] = r[f];
        b -= r[f] * zbar[f];
    }
    *bout = b;
    if (m <= na + 1) return DBL_MAX;
    double e = 0.0;
    for (int a = 0; a < m; ++a) {
        const double* z = Z + (size_t)S->idx[a] * F;
        double p = b;
        for (int f = 0; f < na; ++f) p += w[f] * z[as[f]];
        e += fabs(y[S->idx[a]] - p);
    }
    e /= m;
    const double v = (double)(na + 1);
    return e * ((m + v) / (m - v));
}

/* The model of node t on the candidate attributes `as`, greedily simplified. */
static double m5_node_model(orc_m5_tree* T, int t, const m5_set* S, int F, const double* Z, const double* y,
                            const int* cand, int nc) {
    int as[M5_MAX_TERMS], trial[M5_MAX_TERMS];
    double w[M5_MAX_TERMS], b, wb[M5_MAX_TERMS], bb;
    int na = nc;
    memcpy(as, cand, sizeof(int) * nc);
    double e = m5_fit_lm(S, F, Z, y, as, na, w, &b);
    for (;;) {
        if (na == 0) break;
        double best = DBL_MAX;
        int drop = -1;
        for (int d = 0; d < na; ++d) {
            int nt = 0;
            for (int f = 0; f < na; ++f)
                if (f != d) trial[nt++] = as[f];
            double wt[M5_MAX_TERMS], bt;
            const double et = m5_fit_lm(S, F, Z, y, trial, nt, wt, &bt);
            if (et < best) {
                best = et;
                drop = d;
            }
        }
        if (drop < 0 || !(best <= e)) break;
        for (int f = drop; f < na - 1; ++f) as[f] = as[f + 1];
        --na;
        e = m5_fit_lm(S, F, Z, y, as, na, wb, &bb);
        memcpy(w, wb, sizeof(double) * na);
        b = bb;
    }
    T->nterm[t] = na;
    for (int f = 0; f < na; ++f) {
        T->term_attr[t][f] = as[f];
        T->term_w[t][f] = w[f];
    }
    T->b[t] = b;
    return e;
}

/* Grow the subtree of node t over the instances S (recursive). */
static void m5_grow(orc_m5_tree* T, int t, const m5_set* S, int F, const double* Z, const double* y,
                    double sd_root) {
    T->count[t] = S->m;
    T->attr[t] = -1;
    T->left[t] = T->right[t] = -1;
    double s1 = 0.0, s2 = 0.0;
    for (int a = 0; a < S->m; ++a) {
        s1 += y[S->idx[a]];
        s2 += y[S->idx[a]] * y[S->idx[a]];
    }
    const double sd = m5_sd(S->m, s1, s2);
    if (S->m < M5_MIN_SPLIT || sd <= M5_SD_FRAC * sd_root) return;
    double best = 0.0, bthr = 0.0;
    int battr = -1;
    int ord[M5_MAX_N];
    for (int f = 0; f < F; ++f) {
        /* the node's instances sorted by attribute f, ties by instance index (insertion) */
        for (int a = 0; a < S->m; ++a) {
            const int i = S->idx[a];
            const double v = Z[(size_t)i * F + f];
            int p = a;
            while (p > 0) {
                const int q = ord[p - 1];
                const double u = Z[(size_t)q * F + f];
                if (u > v || (u == v && q > i)) {
                    ord[p] = q;
                    --p;
                } else {
                    break;
                }
            }
            ord[p] = i;
        }
        double l1 = 0.0, l2 = 0.0;
        for (int c = 1; c < S->m; ++c) {
            const double yv = y[ord[c - 1]];
            l1 += yv;
            l2 += yv * yv;
            const double va = Z[(size_t)ord[c - 1] * F + f], vb = Z[(size_t)ord[c] * F + f];
            if (!(va < vb) || c < M5_MIN_SIDE || S->m - c < M5_MIN_SIDE) continue;
            const double sdl = m5_sd(c, l1, l2), sdr = m5_sd(S->m - c, s1 - l1, s2 - l2);
            const double sdr_ = sd - (c * sdl + (S->m - c) * sdr) / S->m;
            if (sdr_ > best) {
                best = sdr_;
                battr = f;
                bthr = (va + vb) * 0.5;
            }
        }
    }
    if (battr < 0) return;
    m5_set L, R;
    L.m = R.m = 0;
    for (int a = 0; a < S->m; ++a) {
        const int i = S->idx[a];
        if (Z[(size_t)i * F + battr] <= bthr) L.idx[L.m++] = i;
        else R.idx[R.m++] = i;
    }
    const int l = T->n_nodes++, r = T->n_nodes++;
    T->attr[t] = battr;
    T->thr[t] = bthr;
    T->left[t] = l;
    T->right[t] = r;
    T->parent[l] = T->parent[r] = t;
    m5_grow(T, l, &L, F, Z, y, sd_root);
    m5_grow(T, r, &R, F, Z, y, sd_root);
}

/* Attributes tested in the subtree of t, as a presence map. */
static void m5_tested(const orc_m5_tree* T, int t, unsigned char* used) {
    if (T->attr[t] < 0) return;
    used[T->attr[t]] = 1;
    m5_tested(T, T->left[t], used);
    m5_tested(T, T->right[t], used);
}

/* Models and pruning of the subtree of t, bottom-up; returns its estimated error. */
static double m5_prune(orc_m5_tree* T, int t, const m5_set* S, int F, const double* Z, const double* y,
                       unsigned char* used) {
    double sub = 0.0;
    if (T->attr[t] >= 0) {
        m5_set L, R;
        L.m = R.m = 0;
        for (int a = 0; a < S->m; ++a) {
            const int i = S->idx[a];
            if (Z[(size_t)i * F + T->attr[t]] <= T->thr[t]) L.idx[L.m++] = i;
            else R.idx[R.m++] = i;
        }
        const double el = m5_prune(T, T->left[t], &L, F, Z, y, used);
        const double er = m5_prune(T, T->right[t], &R, F, Z, y, used);
        sub = (L.m * el + R.m * er) / S->m;
    }
    memset(used, 0, (size_t)F);
    m5_tested(T, t, used);
    int cand[M5_MAX_TERMS], nc = 0;
    for (int f = 0; f < F && nc < M5_MAX_TERMS; ++f)
        if (used[f]) cand[nc++] = f;
    const double e = m5_node_model(T, t, S, F, Z, y, cand, nc);
    if (T->attr[t] >= 0 && !(e <= sub)) {
        T->est[t] = sub;
        return sub;
    }
    T->attr[t] = -1;                    /* a leaf (or pruned to one) */
    T->est[t] = e;
    return e;
}

/* Fit: n instances (n <= 128), rows Zrows [n][F], labels y.  Returns 0, or 1 if n is out of
 * range.  The tree goes to T. */
int orc_m5p_fit(int n, int F, const double* Zrows, const double* y, orc_m5_tree* T) {
    if (n < 1 || n > M5_MAX_N) return 1;
    memset(T, 0, sizeof(*T));
    m5_set S;
    S.m = n;
    for (int a = 0; a < n; ++a) S.idx[a] = a;
    double s1 = 0.0, s2 = 0.0;
    for (int a = 0; a < n; ++a) {
        s1 += y[a];
        s2 += y[a] * y[a];
    }
    T->n_nodes = 1;
    T->parent[0] = -1;
    m5_grow(T, 0, &S, F, Zrows, y, m5_sd(n, s1, s2));
    unsigned char* used = (unsigned char*)malloc((size_t)F);
    m5_prune(T, 0, &S, F, Zrows, y, used);
    free(used);
    return 0;
}

static double m5_model_at(const orc_m5_tree* T, int t, const double* z) {
    double p = T->b[t];
    for (int f = 0; f < T->nterm[t]; ++f) p += T->term_w[t][f] * z[T->term_attr[t][f]];
    return p;
}

double orc_m5p_predict(const orc_m5_tree* T, const double* z) {
    int t = 0;
    while (T->attr[t] >= 0) t = z[T->attr[t]] <= T->thr[t] ? T->left[t] : T->right[t];
    double p = m5_model_at(T, t, z);
    while (T->parent[t] >= 0) {
        const int u = T->parent[t];
        const double nc = (double)T->count[t];
        p = (nc * p + M5_SMOOTH_K * m5_model_at(T, u, z)) / (nc + M5_SMOOTH_K);
        t = u;
    }
    return p;
}

int orc_m5p_tree_bytes(void) { return (int)sizeof(orc_m5_tree); }
int orc_m5p_fit_tree(int n, int F, const double* Zrows, const double* y, void* T) {
    return orc_m5p_fit(n, F, Zrows, y, (orc_m5_tree*)T);
}
double orc_m5p_predict_tree(const void* T, const double* z) { return orc_m5p_predict((const orc_m5_tree*)T, z); }

/* One-shot helper for tests: fit on (Zrows, y) and predict for the rows of Zt [nt][F]. */
int orc_m5p_fit_predict(int n, int F, const double* Zrows, const double* y, int nt, const double* Zt,
                        double* pred, int* n_leaves, int* n_nodes) {
    orc_m5_tree* T = (orc_m5_tree*)malloc(sizeof(orc_m5_tree));
    const int st = orc_m5p_fit(n, F, Zrows, y, T);
    if (st == 0) {
        for (int t = 0; t < nt; ++t) pred[t] = orc_m5p_predict(T, Zt + (size_t)t * F);
        int leaves = 0, reach = 0;
        /* nodes reachable after pruning */
        int stack[M5_MAX_NODES], sp = 0;
        stack[sp++] = 0;
        while (sp) {
            const int u = stack[--sp];
            ++reach;
            if (T->attr[u] < 0) ++leaves;
            else {
                stack[sp++] = T->left[u];
                stack[sp++] = T->right[u];
            }
        }
        if (n_leaves) *n_leaves = leaves;
        if (n_nodes) *n_nodes = reach;
    }
    free(T);
    return st;
}
