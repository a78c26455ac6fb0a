// Table 2 transfer (Sec. 5): the fits of each problem's training group of runs (one block per
// problem and optimization), then the predictions for its test program, ranking and scoring
// (one block per problem).
#include <float.h>

#include "rank_row.cuh"

namespace {

// ====================================================================== transfer (Table 2)
// A problem q trains on a group of runs: every before/after pair of every run, run by run in
// ascending before slot, a pair never spanning two runs.  The group's versions form one list
// of N (rs_group_layout); KA[q] is their Gram, Kx[q][t][u] the block between test row t and
// version u (dot products; squared distances for IBK).
// Ridge: the bordered dual system of each optimization, M = KA(pairs) + lambda I = L D L^T,
// then b and alpha as in the batched solvers, and the prediction b + sum_a alpha_a Kx[t][u_a].
// IBK: the mean label of the kIbkK pairs nearest to t.  Candidates: outside t's mask (all six
// with RS_RANK_ALL) and inside opt_mask; ranking, threshold, top-k and scoring as in the rank
// pass with the test program's own times.
constexpr int kTrPairs = RS_MAXPAIRS * RS_MAXRUNS;   // pairs of one fit
constexpr int kTrRows = RS_MAXV * RS_MAXRUNS;        // versions of one group
constexpr int kTrThreads = 128;
constexpr int kTrCoef = kTrPairs + 1;                // b, alpha[kTrPairs] per fit in the workspace

// The training group of a problem in shared memory: its versions' masks and log times, and
// the slot of each mask within each run (-1 if absent).
struct GroupSmem {
    double lt[kTrRows];
    uint8_t msk[kTrRows];
    int8_t slot[RS_MAXRUNS][RS_MAXV];
};

__device__ void load_group(GroupSmem& G, const int64_t* __restrict__ a_row, const uint8_t* __restrict__ a_masks,
                           const double* __restrict__ a_lt, int64_t g0, const int (&start)[RS_MAXRUNS + 1], int N) {
    for (int e = threadIdx.x; e < RS_MAXRUNS * RS_MAXV; e += blockDim.x) G.slot[e / RS_MAXV][e % RS_MAXV] = -1;
    for (int u = threadIdx.x; u < N; u += blockDim.x) {
        int r = 0;
        while (u >= start[r + 1]) ++r;
        const int64_t row = a_row[g0 + r] + (u - start[r]);
        G.msk[u] = a_masks[row] & 63;
        G.lt[u] = a_lt[row];
    }
    __syncthreads();
    for (int u = threadIdx.x; u < N; u += blockDim.x) {
        int r = 0;
        while (u >= start[r + 1]) ++r;
        G.slot[r][G.msk[u]] = (int8_t)(u - start[r]);
    }
    __syncthreads();
}

// The pairs of optimization j (one thread): group version of each before side, and labels.
// Returns their number; more than kTrPairs (only possible with repeated masks) is reported.
__device__ int build_pairs(const GroupSmem& G, int j, int R, const int (&start)[RS_MAXRUNS + 1], uint16_t* pu,
                           double* yl, int* dstatus, int q) {
    int np = 0;
    for (int r = 0; r < R; ++r)
        for (int u = start[r]; u < start[r + 1]; ++u) {
            const int m = G.msk[u];
            if ((m >> j) & 1) continue;
            const int w = G.slot[r][m | (1 << j)];
            if (w < 0) continue;
            if (np == kTrPairs) {
                rs_dev_flag(dstatus, RS_EDATA, q);
                continue;
            }
            pu[np] = (uint16_t)u;
            yl[np] = G.lt[u] - G.lt[start[r] + w];
            ++np;
        }
    return np;
}

struct M5Tree;

struct TransferArgs {
    const int64_t* group_off;
    int max_runs, stat_stride;
    int64_t n_runs;
    const int64_t* a_row;
    const int32_t* a_fw;
    const uint8_t* a_masks;
    const double* a_lt;
    const int64_t* b_row;
    const int32_t* b_fw;
    const uint8_t* b_masks;
    const double* b_lt;
    const double* KA;
    const double* Kx;
    int ld;
    double lambda;
    double* coef;                        // [Q][6][kTrCoef] ridge fits (written by the fit kernel)
    uint8_t* fst;                        // [Q][6] their status
    int ibk, opt_mask, rank_all;
    int m5p;                             // the M5P model tree instead of ridge
    M5Tree* trees;                       // [Q][6] M5P trees
    const double* ZA;                    // standardized training group rows (M5P fits)
    const int64_t* a_xo;
    const double* ZB;                    // standardized test rows (M5P predictions)
    const int64_t* b_xo;
    uint8_t* fit_status;
    RankPassArgs r;                      // k, ktau, flags (without RS_RANK_ALL), outputs, counters
};

// Reciprocal of a nonzero finite double of either sign (rcp_newton on its magnitude).
__device__ __forceinline__ double rcp_newton_any(double d) {
    return d < 0.0 ? -rcp_newton(-d) : rcp_newton(d);
}

// One block per (problem, optimization): the ridge fit of that optimization's pairs.  The
// factor lives in shared memory (nmax rows of nmax + 1 doubles); right-looking LDL^T whose
// trailing update of each step is spread over all threads (16 row groups x 8 column lanes),
// reciprocal pivots from rcp_newton kept for the solves, then the two forward solves and the
// back solve of the bordered system, one thread per row.
__global__ void __launch_bounds__(kTrThreads)
transfer_fit_kernel(const TransferArgs a, int nmax) {
    extern __shared__ __align__(16) double fsm[];
    __shared__ GroupSmem G;
    __shared__ uint16_t pu[kTrPairs];
    __shared__ double yl[kTrPairs];
    __shared__ int np_s;
    __shared__ double bval;
    __shared__ double red[8];
    const int q = blockIdx.x, j = blockIdx.y, tid = threadIdx.x;
    const int ldm = nmax + 1;
    double* M = fsm;
    double* col = M + (size_t)nmax * ldm;
    double* lrow = col + nmax;
    double* ty = lrow + nmax;
    double* t1 = ty + nmax;
    double* dinv = t1 + nmax;
    int start[RS_MAXRUNS + 1], F = 0;
    const int N = rs_group_layout(q, a.group_off, a.max_runs, a.n_runs, a.a_row, a.a_fw, a.b_fw, a.stat_stride, start, F);
    if (N < 0 || N > a.ld) return;                 // reported by the predict / rank kernel
    const int64_t g0 = a.group_off[q];
    const int R = (int)(a.group_off[q + 1] - g0);
    load_group(G, a.a_row, a.a_masks, a.a_lt, g0, start, N);
    if (tid == 0) np_s = build_pairs(G, j, R, start, pu, yl, nullptr, q);
    __syncthreads();
    const int n = np_s;
    double* out = a.coef + ((int64_t)q * RS_NOPT + j) * kTrCoef;
    uint8_t* st_out = a.fst + (int64_t)q * RS_NOPT + j;
    if (n == 0 || n > nmax) {                      // n > nmax: more pairs than the hint allowed
        if (tid == 0) *st_out = n == 0 ? RS_FIT_EMPTY : RS_FIT_NOTPD;
        return;
    }
    if (n == 1) {                                  // one pair: alpha = 0, b = its label
        if (tid == 0) {
            out[0] = yl[0];
            out[1] = 0.0;
            *st_out = finite_bits(yl[0]) ? RS_FIT_OK : RS_FIT_NONFINITE;
        }
        return;
    }
    const double* KAq = a.KA + (int64_t)q * a.ld * a.ld;
    for (int e = tid; e < n * n; e += kTrThreads) {
        const int i = e / n, c = e - i * n;
        if (c <= i) M[i * ldm + c] = __ldg(KAq + (int64_t)pu[i] * a.ld + pu[c]) + (i == c ? a.lambda : 0.0);
    }
    __syncthreads();
    const int ty8 = tid >> 3, tx8 = tid & 7;
    int st = RS_FIT_OK;
    for (int k = 0; k < n; ++k) {
        const double d = M[k * ldm + k];
        if (!pos_finite(d)) {                      // every thread read the same pivot
            st = RS_FIT_NOTPD;
            break;
        }
        const double di = rcp_newton(d);
        if (tid == 0) dinv[k] = di;
        for (int i = k + 1 + tid; i < n; i += kTrThreads) {
            const double c = M[i * ldm + k];
            col[i] = c;
            lrow[i] = c * di;
            M[i * ldm + k] = c * di;
        }
        __syncthreads();
        for (int i = k + 1 + ty8; i < n; i += 16) {
            const double l = lrow[i];
            for (int c = k + 1 + tx8; c <= i; c += 8) M[i * ldm + c] = fma(-l, col[c], M[i * ldm + c]);
        }
        __syncthreads();
    }
    if (st == RS_FIT_OK) {
        if (tid < n) {                             // L t = rhs, two right-hand sides
            ty[tid] = yl[tid];
            t1[tid] = 1.0;
        }
        __syncthreads();
        for (int k = 0; k < n - 1; ++k) {
            if (tid > k && tid < n) {
                const double l = M[tid * ldm + k];
                ty[tid] = fma(-l, ty[k], ty[tid]);
                t1[tid] = fma(-l, t1[k], t1[tid]);
            }
            __syncthreads();
        }
        // num = t_1^T D^-1 t_y, den = t_1^T D^-1 t_1: per-thread terms, warp trees, then the
        // four warps' sums in order
        double pn = 0.0, pd = 0.0;
        if (tid < n) {
            const double sc = t1[tid] * dinv[tid];
            pn = sc * ty[tid];
            pd = sc * t1[tid];
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            pn += __shfl_xor_sync(0xffffffffu, pn, o);
            pd += __shfl_xor_sync(0xffffffffu, pd, o);
        }
        if ((tid & 31) == 0) {
            red[tid >> 5] = pn;
            red[4 + (tid >> 5)] = pd;
        }
        __syncthreads();
        if (tid == 0) bval = ((red[0] + red[1]) + (red[2] + red[3])) * rcp_newton_any(((red[4] + red[5]) + (red[6] + red[7])));
        __syncthreads();
        const double b = bval;
        if (tid < n) ty[tid] = fma(-b, t1[tid], ty[tid]) * dinv[tid];
        __syncthreads();
        for (int k = n - 1; k > 0; --k) {          // L^T alpha = D^-1 (t_y - b t_1)
            if (tid < k) ty[tid] = fma(-M[k * ldm + tid], ty[k], ty[tid]);
            __syncthreads();
        }
        bool fin = true;
        if (tid < n) {
            out[1 + tid] = ty[tid];
            fin = finite_bits(ty[tid]);
        }
        if (tid == 0) out[0] = b;
        st = __syncthreads_and(fin) && finite_bits(b) ? RS_FIT_OK : RS_FIT_NONFINITE;
    }
    if (tid == 0) *st_out = (uint8_t)st;
}

// ====================================================================== M5P (Sec. 3.4)
// The model tree of each (problem, optimization), after the M5' description: grow by the
// standard deviation reduction (SDR), a linear model at every node on the attributes tested
// in its subtree as pruned so far (children are modelled and pruned first), simplified by
// greedy elimination, bottom-up pruning by estimated error, and smoothing on the way up at
// prediction time (k = 15).
constexpr int kM5MaxN = kTrPairs;                 // instances of one fit
constexpr int kM5MaxNodes = 2 * kM5MaxN - 1;
constexpr int kM5MaxTerms = 64;
constexpr int kM5MaxFeat = 256;                   // attributes (one thread each in the split search)
constexpr int kM5Threads = 256;
constexpr int kM5Ld = kM5MaxTerms + 1;
constexpr double kM5SdFrac = 0.05, kM5Smooth = 15.0, kM5Ridge = 1e-8;

struct M5Tree {
    int n_nodes;
    int count[kM5MaxNodes];
    int nterm[kM5MaxNodes];
    int16_t attr[kM5MaxNodes], left[kM5MaxNodes], right[kM5MaxNodes], parent[kM5MaxNodes];
    double thr[kM5MaxNodes], b[kM5MaxNodes];
    int16_t term_attr[kM5MaxNodes][kM5MaxTerms];
    double term_w[kM5MaxNodes][kM5MaxTerms];
};

struct M5Smem {
    union {                                       // the growing pass, then the models' pass
        struct {
            uint8_t sorted[kM5MaxFeat][kM5MaxN];  // per attribute: instances in (value, index) order
            uint8_t scratch[kM5Threads][kM5MaxN];
        } gr;
        struct {
            double G[kM5MaxTerms * kM5Ld];        // centred normal equations of the node's candidates
            double H[kM5MaxTerms * kM5Ld];        // inverse of the current subset's system
        } mo;
    };
    double colk[kM5MaxTerms], rowk[kM5MaxTerms];
    double zbar[kM5MaxTerms], r[kM5MaxTerms], w[kM5MaxTerms], cand_err[kM5MaxTerms];
    double res[kM5MaxN];
    double y[kM5MaxN];
    const double* zp[kM5MaxN];                    // each instance's standardized row
    double thr[kM5MaxNodes], est[kM5MaxNodes];
    unsigned long long tested[kM5MaxNodes][kM5MaxFeat / 64];
    int16_t attr[kM5MaxNodes], left[kM5MaxNodes], right[kM5MaxNodes];
    uint8_t lo[kM5MaxNodes], hi[kM5MaxNodes];
    uint8_t ids[kM5MaxN];
    uint8_t side[kM5MaxN];
    uint8_t sel[kM5MaxTerms];                     // current subset: positions in the candidate list
    int16_t cand[kM5MaxTerms];
    double red_v[kM5Threads / 32];
    int red_i[kM5Threads / 32];
    int stack_node[kM5MaxNodes], stack_lo[kM5MaxNodes], stack_hi[kM5MaxNodes];
    int sp, nn, cur, cur_lo, cur_hi, ncand, nsel, split_attr, drop;
    double split_thr, sd_root, e_cur, bval;
};

// The standard deviation from a count, sum and sum of squares: sqrt(max(0, (s2 - s1 s1 / c) / c)),
// with one rounding per operation (the reference's arithmetic).
__device__ __forceinline__ double m5_sd(int c, double s1, double s2) {
    const double cd = (double)c;
    const double v = __ddiv_rn(__dsub_rn(s2, __ddiv_rn(__dmul_rn(s1, s1), cd)), cd);
    return __dsqrt_rn(v > 0.0 ? v : 0.0);
}

// In-place inverse of the nb x nb leading block of M (row stride kM5Ld) by Gauss-Jordan
// elimination without pivoting (the systems are symmetric positive definite).  Block-wide.
__device__ void m5_invert(M5Smem& S, double* M, int nb) {
    const int tid = threadIdx.x;
    for (int k = 0; k < nb; ++k) {
        const double piv = 1.0 / M[k * kM5Ld + k];
        for (int i = tid; i < nb; i += kM5Threads) {
            S.colk[i] = M[i * kM5Ld + k];
            S.rowk[i] = M[k * kM5Ld + i] * piv;
        }
        __syncthreads();
        for (int e = tid; e < nb * nb; e += kM5Threads) {
            const int i = e / nb, j = e - i * nb;
            if (i == k && j == k) M[k * kM5Ld + k] = piv;
            else if (i == k) M[k * kM5Ld + j] = S.rowk[j];
            else if (j == k) M[i * kM5Ld + k] = -S.colk[i] * piv;
            else M[i * kM5Ld + j] = fma(-S.colk[i], S.rowk[j], M[i * kM5Ld + j]);
        }
        __syncthreads();
    }
}

// Estimated error of a model (b, w on the selected candidates) over the node's instances:
// mean |y - prediction| * (m + v) / (m - v), v = terms + 1; DBL_MAX when m <= v.  One warp.
__device__ double m5_warp_err(const M5Smem& S, int lo, int m, const double* w, double b, int nsel,
                              const uint8_t* selpos, int skip) {
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int a = lane; a < m; a += 32) {
        const int i = S.ids[lo + a];
        const double* z = S.zp[i];
        double p = b;
        for (int q = 0; q < nsel; ++q) {
            if (q == skip) continue;
            p = fma(w[q], __ldg(z + S.cand[selpos[q]]), p);
        }
        acc += fabs(S.y[i] - p);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const int v = nsel - (skip >= 0 ? 1 : 0) + 1;
    if (m <= v) return DBL_MAX;
    return acc / m * ((double)(m + v) / (double)(m - v));
}

__global__ void __launch_bounds__(kM5Threads, 1)
m5p_fit_kernel(const TransferArgs a) {
    extern __shared__ __align__(16) unsigned char m5sm[];
    M5Smem& S = *reinterpret_cast<M5Smem*>(m5sm);
    __shared__ GroupSmem G;
    __shared__ uint16_t pu[kTrPairs];
    __shared__ double yl[kTrPairs];
    __shared__ int np_s;
    const int q = blockIdx.x, j = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kM5Threads / 32;
    int start[RS_MAXRUNS + 1], F = 0;
    const int N = rs_group_layout(q, a.group_off, a.max_runs, a.n_runs, a.a_row, a.a_fw, a.b_fw, a.stat_stride, start, F);
    if (N < 0 || N > a.ld || F > kM5MaxFeat) return;   // reported by the predict / rank kernel
    const int64_t g0 = a.group_off[q];
    const int R = (int)(a.group_off[q + 1] - g0);
    load_group(G, a.a_row, a.a_masks, a.a_lt, g0, start, N);
    if (tid == 0) np_s = build_pairs(G, j, R, start, pu, yl, nullptr, q);
    __syncthreads();
    const int n = np_s;
    M5Tree* T = a.trees + ((int64_t)q * RS_NOPT + j);
    uint8_t* st_out = a.fst + (int64_t)q * RS_NOPT + j;
    if (n == 0) {
        if (tid == 0) *st_out = RS_FIT_EMPTY;
        return;
    }
    for (int i = tid; i < n; i += kM5Threads) {
        const int u = pu[i];
        int r = 0;
        while (u >= start[r + 1]) ++r;
        S.zp[i] = a.ZA + a.a_xo[g0 + r] + (int64_t)(u - start[r]) * F;
        S.y[i] = yl[i];
        S.ids[i] = (uint8_t)i;
    }
    __syncthreads();
    // presort: attribute f's instances by (value, index)
    for (int f = tid; f < F; f += kM5Threads) {
        uint8_t* o = S.gr.sorted[f];
        for (int i = 0; i < n; ++i) {
            const double v = __ldg(S.zp[i] + f);
            int p = i;
            while (p > 0) {
                const int w = o[p - 1];
                const double u = __ldg(S.zp[w] + f);
                if (u > v || (u == v && w > i)) {
                    o[p] = (uint8_t)w;
                    --p;
                } else {
                    break;
                }
            }
            o[p] = (uint8_t)i;
        }
    }
    if (tid == 0) {
        S.nn = 1;
        S.sp = 1;
        S.stack_node[0] = 0;
        S.stack_lo[0] = 0;
        S.stack_hi[0] = n;
        double s1 = 0.0, s2 = 0.0;
        for (int i = 0; i < n; ++i) {
            s1 = __dadd_rn(s1, S.y[i]);
            s2 = __dadd_rn(s2, __dmul_rn(S.y[i], S.y[i]));
        }
        S.sd_root = m5_sd(n, s1, s2);
    }
    __syncthreads();
    // ---- grow (depth first, left child first: the reference's node numbering).  Thread 0 pops
    // the next node; every path through the body ends at a barrier before the next pop.
    for (;;) {
        if (tid == 0) {
            if (S.sp > 0) {
                --S.sp;
                S.cur = S.stack_node[S.sp];
                S.cur_lo = S.stack_lo[S.sp];
                S.cur_hi = S.stack_hi[S.sp];
            } else {
                S.cur = -1;
            }
        }
        __syncthreads();
        const int t = S.cur, lo = S.cur_lo, hi = S.cur_hi, m = hi - lo;
        if (t < 0) break;
        if (tid == 0) {
            S.attr[t] = -1;
            S.lo[t] = (uint8_t)lo;
            S.hi[t] = (uint8_t)hi;
        }
        // the node's label sums in instance order
        double s1 = 0.0, s2 = 0.0;
        for (int a2 = lo; a2 < hi; ++a2) {
            const double yv = S.y[S.ids[a2]];
            s1 = __dadd_rn(s1, yv);
            s2 = __dadd_rn(s2, __dmul_rn(yv, yv));
        }
        const double sd = m5_sd(m, s1, s2);
        if (m < 4 || sd <= __dmul_rn(kM5SdFrac, S.sd_root)) {
            __syncthreads();
            continue;
        }
        // split search: one thread per attribute, candidates in sorted order
        double best = 0.0, bthr = 0.0;
        int battr = -1;
        for (int f = tid; f < F; f += kM5Threads) {
            const uint8_t* o = S.gr.sorted[f];
            double l1 = 0.0, l2 = 0.0;
            for (int c = 1; c < m; ++c) {
                const int ia = o[lo + c - 1], ib = o[lo + c];
                const double yv = S.y[ia];
                l1 = __dadd_rn(l1, yv);
                l2 = __dadd_rn(l2, __dmul_rn(yv, yv));
                const double va = __ldg(S.zp[ia] + f), vb = __ldg(S.zp[ib] + f);
                if (!(va < vb) || c < 2 || m - c < 2) continue;
                const double sdl = m5_sd(c, l1, l2), sdr = m5_sd(m - c, __dsub_rn(s1, l1), __dsub_rn(s2, l2));
                const double red = __dsub_rn(sd, __ddiv_rn(__dadd_rn(__dmul_rn((double)c, sdl),
                                                                     __dmul_rn((double)(m - c), sdr)),
                                                           (double)m));
                if (red > best) {
                    best = red;
                    battr = f;
                    bthr = __dmul_rn(__dadd_rn(va, vb), 0.5);
                }
            }
        }
        // block argmax: largest SDR, ties to the lower attribute
#pragma unroll
        for (int o2 = 16; o2 >= 1; o2 >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o2);
            const int oa = __shfl_xor_sync(0xffffffffu, battr, o2);
            const double ot = __shfl_xor_sync(0xffffffffu, bthr, o2);
            if (oa >= 0 && (battr < 0 || ob > best || (ob == best && oa < battr))) {
                best = ob;
                battr = oa;
                bthr = ot;
            }
        }
        if (lane == 0) {
            S.red_v[warp] = best;
            S.red_i[warp] = battr;
            S.colk[warp] = bthr;
        }
        __syncthreads();
        if (tid == 0) {
            double bb = 0.0, bt = 0.0;
            int ba = -1;
            for (int w2 = 0; w2 < nwarps; ++w2) {
                const int oa = S.red_i[w2];
                if (oa >= 0 && (ba < 0 || S.red_v[w2] > bb || (S.red_v[w2] == bb && oa < ba))) {
                    bb = S.red_v[w2];
                    ba = oa;
                    bt = S.colk[w2];
                }
            }
            S.split_attr = ba;
            S.split_thr = bt;
        }
        __syncthreads();
        const int sa = S.split_attr;
        if (sa < 0) {                              // no admissible split: a leaf (uniform)
            __syncthreads();
            continue;
        }
        const double sthr = S.split_thr;
        for (int a2 = lo + tid; a2 < hi; a2 += kM5Threads) {
            const int i = S.ids[a2];
            S.side[i] = __ldg(S.zp[i] + sa) <= sthr ? 0 : 1;
        }
        __syncthreads();
        // stable partition of the node's instance list and of every attribute's sorted list
        int nl = 0;
        for (int f = tid; f < F + 1; f += kM5Threads) {
            uint8_t* o = f < F ? S.gr.sorted[f] : S.ids;
            uint8_t* sc = S.gr.scratch[tid];
            int k = 0;
            for (int a2 = lo; a2 < hi; ++a2)
                if (S.side[o[a2]] == 0) sc[k++] = o[a2];
            nl = k;
            for (int a2 = lo; a2 < hi; ++a2)
                if (S.side[o[a2]] == 1) sc[k++] = o[a2];
            for (int a2 = 0; a2 < m; ++a2) o[lo + a2] = sc[a2];
        }
        __syncthreads();
        if (tid == 0) {
            int cnt = 0;
            for (int a2 = lo; a2 < hi; ++a2) cnt += S.side[S.ids[a2]] == 0;
            const int l = S.nn, r = S.nn + 1;
            S.nn += 2;
            S.attr[t] = (int16_t)sa;
            S.thr[t] = sthr;
            S.left[t] = (int16_t)l;
            S.right[t] = (int16_t)r;
            T->parent[l] = T->parent[r] = (int16_t)t;
            S.stack_node[S.sp] = r;
            S.stack_lo[S.sp] = lo + cnt;
            S.stack_hi[S.sp] = hi;
            ++S.sp;
            S.stack_node[S.sp] = l;
            S.stack_lo[S.sp] = lo;
            S.stack_hi[S.sp] = lo + cnt;
            ++S.sp;
        }
        (void)nl;
        __syncthreads();
    }
    const int nn = S.nn;
    // ---- models and pruning, children before parents (children have larger node numbers)
    for (int t = nn - 1; t >= 0; --t) {
        const int lo = S.lo[t], m = S.hi[t] - S.lo[t];
        const bool internal = S.attr[t] >= 0;
        if (tid < kM5MaxFeat / 64) {
            unsigned long long bits = 0;
            if (internal) {
                bits = S.tested[S.left[t]][tid] | S.tested[S.right[t]][tid];
                if (S.attr[t] / 64 == tid) bits |= 1ull << (S.attr[t] % 64);
            }
            S.tested[t][tid] = bits;
        }
        __syncthreads();
        if (tid == 0) {
            int nc = 0;
            for (int f = 0; f < F && nc < kM5MaxTerms; ++f)
                if ((S.tested[t][f / 64] >> (f % 64)) & 1ull) S.cand[nc++] = (int16_t)f;
            S.ncand = nc;
            S.nsel = nc;
            for (int k = 0; k < nc; ++k) S.sel[k] = (uint8_t)k;
            double yb = 0.0;
            for (int a2 = 0; a2 < m; ++a2) yb += S.y[S.ids[lo + a2]];
            S.bval = yb / m;                       // the label mean, for now
        }
        __syncthreads();
        const int nc = S.ncand;
        const double ybar = S.bval;
        for (int f = tid; f < nc; f += kM5Threads) {
            double s = 0.0;
            for (int a2 = 0; a2 < m; ++a2) s += __ldg(S.zp[S.ids[lo + a2]] + S.cand[f]);
            S.zbar[f] = s / m;
        }
        __syncthreads();
        for (int e = tid; e < nc * (nc + 1); e += kM5Threads) {
            const int f = e / (nc + 1), g = e - f * (nc + 1);
            double s = 0.0;
            if (g < nc) {
                if (g > f) continue;
                for (int a2 = 0; a2 < m; ++a2) {
                    const double* z = S.zp[S.ids[lo + a2]];
                    s += (__ldg(z + S.cand[f]) - S.zbar[f]) * (__ldg(z + S.cand[g]) - S.zbar[g]);
                }
                S.mo.G[f * kM5Ld + g] = s + (f == g ? kM5Ridge : 0.0);
                S.mo.G[g * kM5Ld + f] = s + (f == g ? kM5Ridge : 0.0);
            } else {
                for (int a2 = 0; a2 < m; ++a2) {
                    const int i = S.ids[lo + a2];
                    s += (__ldg(S.zp[i] + S.cand[f]) - S.zbar[f]) * (S.y[i] - ybar);
                }
                S.r[f] = s;
            }
        }
        __syncthreads();
        // greedy elimination
        for (;;) {
            const int ns = S.nsel;
            for (int e = tid; e < ns * ns; e += kM5Threads) {
                const int i = e / ns, k = e - i * ns;
                S.mo.H[i * kM5Ld + k] = S.mo.G[S.sel[i] * kM5Ld + S.sel[k]];
            }
            __syncthreads();
            m5_invert(S, S.mo.H, ns);
            for (int i = tid; i < ns; i += kM5Threads) {
                double s = 0.0;
                for (int k = 0; k < ns; ++k) s = fma(S.mo.H[i * kM5Ld + k], S.r[S.sel[k]], s);
                S.w[i] = s;
            }
            __syncthreads();
            if (tid == 0) {
                double b = ybar;
                for (int i = 0; i < ns; ++i) b -= S.w[i] * S.zbar[S.sel[i]];
                S.rowk[0] = b;                     // the model's intercept
            }
            __syncthreads();
            if (warp == 0) {
                const double e_full = m5_warp_err(S, lo, m, S.w, S.rowk[0], ns, S.sel, -1);
                if (lane == 0) S.e_cur = e_full;
            }
            // drop-one candidates: w' = w - H[:, d] w_d / H_dd, one warp each
            for (int d = warp; d < ns; d += nwarps) {
                const double fac = S.w[d] / S.mo.H[d * kM5Ld + d];
                double wd[kM5MaxTerms];
                double b = ybar;
                for (int i = 0; i < ns; ++i) {
                    wd[i] = i == d ? 0.0 : fma(-S.mo.H[i * kM5Ld + d], fac, S.w[i]);
                    if (i != d) b -= wd[i] * S.zbar[S.sel[i]];
                }
                const double ed = m5_warp_err(S, lo, m, wd, b, ns, S.sel, d);
                if (lane == 0) S.cand_err[d] = ed;
            }
            __syncthreads();
            if (tid == 0) {
                double bestd = DBL_MAX;
                int drop = -1;
                for (int d = 0; d < ns; ++d)
                    if (S.cand_err[d] < bestd) {
                        bestd = S.cand_err[d];
                        drop = d;
                    }
                S.drop = (ns > 0 && drop >= 0 && bestd <= S.e_cur) ? drop : -1;
                if (S.drop >= 0) {
                    for (int k = S.drop; k < ns - 1; ++k) S.sel[k] = S.sel[k + 1];
                    S.nsel = ns - 1;
                }
            }
            __syncthreads();
            if (S.drop < 0) break;
        }
        // the node's model and the pruning decision
        if (tid == 0) {
            const int ns = S.nsel;
            T->nterm[t] = ns;
            for (int k = 0; k < ns; ++k) {
                T->term_attr[t][k] = S.cand[S.sel[k]];
                T->term_w[t][k] = S.w[k];
            }
            T->b[t] = S.rowk[0];
            T->count[t] = m;
            const double e = S.e_cur;
            double keep = DBL_MAX;
            if (internal) {
                const int l = S.left[t], r = S.right[t];
                const int ml = S.hi[l] - S.lo[l], mr = S.hi[r] - S.lo[r];
                keep = (ml * S.est[l] + mr * S.est[r]) / m;
            }
            if (internal && !(e <= keep)) {
                S.est[t] = keep;
            } else {                               // a leaf: its parent's candidates get no test
                S.attr[t] = -1;                    // from here down
                S.est[t] = e;
                for (int k = 0; k < kM5MaxFeat / 64; ++k) S.tested[t][k] = 0;
            }
        }
        __syncthreads();
    }
    for (int t = tid; t < nn; t += kM5Threads) {
        T->attr[t] = S.attr[t];
        T->thr[t] = S.thr[t];
        T->left[t] = S.left[t];
        T->right[t] = S.right[t];
    }
    if (tid == 0) {
        T->n_nodes = nn;
        T->parent[0] = -1;
        *st_out = RS_FIT_OK;
    }
}

// The M5P prediction for one test vector: the leaf's model, then smoothing with every
// ancestor's model on the way up, p = (n_c p + k q) / (n_c + k).
__device__ double m5_predict(const M5Tree* __restrict__ T, const double* __restrict__ z) {
    auto model = [&](int t) {
        double p = T->b[t];
        for (int k = 0; k < T->nterm[t]; ++k) p = fma(T->term_w[t][k], __ldg(z + T->term_attr[t][k]), p);
        return p;
    };
    int t = 0;
    while (T->attr[t] >= 0) t = __ldg(z + T->attr[t]) <= T->thr[t] ? T->left[t] : T->right[t];
    double p = model(t);
    while (T->parent[t] >= 0) {
        const int u = T->parent[t];
        const double nc = (double)T->count[t];
        p = (nc * p + kM5Smooth * model(u)) / (nc + kM5Smooth);
        t = u;
    }
    return p;
}

// ibk_nearest_mean for a list of n > kIbkK pairs (n up to kTrPairs): the chosen labels are
// summed in ascending pair index.
__device__ __forceinline__ double ibk_nearest_mean_n(int n, const double* __restrict__ Dt, const uint16_t* pu,
                                                     const double* yl) {
    unsigned long long kd[kIbkK];
    int kq[kIbkK];
#pragma unroll
    for (int i = 0; i < kIbkK; ++i) {
        kd[i] = ~0ull;
        kq[i] = 0;
    }
    for (int q = 0; q < n; ++q) ibk_insert(kd, kq, (unsigned long long)__double_as_longlong(__ldg(Dt + pu[q])), q);
    for (int i = 1; i < kIbkK; ++i)          // indices ascending
        for (int m = i; m > 0 && kq[m - 1] > kq[m]; --m) {
            const int x = kq[m];
            kq[m] = kq[m - 1];
            kq[m - 1] = x;
        }
    double sum = 0.0;
    for (int i = 0; i < kIbkK; ++i) sum += yl[kq[i]];
    return sum / (double)kIbkK;
}

// One block per problem, one thread per version t of the test program: the pairs of the six
// optimizations (the fits' order), the predictions (ridge: the fits of transfer_fit_kernel;
// IBK: the neighbour lists), and rank_row.
struct RankSmem {
    GroupSmem G;
    double yl[RS_NOPT][kTrPairs];
    double lt_b[RS_MAXV];
    uint16_t pu[RS_NOPT][kTrPairs];
    uint8_t msk_b[RS_MAXV];
    int8_t slot_b[RS_MAXV];
    int np[RS_NOPT], st[RS_NOPT];
};

__global__ void __launch_bounds__(RS_MAXV)
transfer_rank_kernel(const TransferArgs a) {
    extern __shared__ __align__(16) unsigned char tsm[];
    RankSmem& S = *reinterpret_cast<RankSmem*>(tsm);
    const int q = blockIdx.x, tid = threadIdx.x;
    int start[RS_MAXRUNS + 1], F = 0;
    const int N = rs_group_layout(q, a.group_off, a.max_runs, a.n_runs, a.a_row, a.a_fw, a.b_fw, a.stat_stride, start, F);
    const int64_t rb = a.b_row[q];
    const int VB = (int)(a.b_row[q + 1] - rb);
    if (N < 0 || N > a.ld || VB < 1 || VB > RS_MAXV) {
        if (tid == 0) rs_dev_flag(a.r.dstatus, RS_EDATA, q);
        return;
    }
    const int64_t g0 = a.group_off[q];
    const int R = (int)(a.group_off[q + 1] - g0);
    S.slot_b[tid] = -1;
    if (tid < VB) {
        S.msk_b[tid] = a.b_masks[rb + tid] & 63;
        S.lt_b[tid] = a.b_lt[rb + tid];
    }
    load_group(S.G, a.a_row, a.a_masks, a.a_lt, g0, start, N);
    if (tid < VB) S.slot_b[S.msk_b[tid]] = (int8_t)tid;
    if (tid < RS_NOPT) {
        const int j = tid;
        const int np = build_pairs(S.G, j, R, start, S.pu[j], S.yl[j], a.r.dstatus, q);
        S.np[j] = np;
        S.st[j] = a.ibk ? (np > 0 ? RS_FIT_OK : RS_FIT_EMPTY) : a.fst[(int64_t)q * RS_NOPT + j];
        if (a.m5p && np > kM5MaxN) S.st[j] = RS_FIT_NOTPD;
    }
    __syncthreads();
    RankTally c;
    const int t = tid;
    if (t < VB) {
        const int mt = S.msk_b[t];
        const uint32_t info = row_summary(t, VB, S.msk_b, S.lt_b, S.slot_b);
        const int candm = (a.rank_all ? 63 : (~mt & 63)) & a.opt_mask;
        int okm = 0;
#pragma unroll
        for (int j = 0; j < RS_NOPT; ++j) okm |= (S.st[j] == RS_FIT_OK) << j;
        const double* Kt = a.Kx + ((int64_t)q * RS_MAXV + t) * a.ld;
        double pred[RS_NOPT];
#pragma unroll
        for (int j = 0; j < RS_NOPT; ++j) {
            pred[j] = 0.0;
            if (!(((candm & okm) >> j) & 1)) continue;
            const int n = S.np[j];
            if (a.m5p) {
                pred[j] = m5_predict(a.trees + ((int64_t)q * RS_NOPT + j), a.ZB + a.b_xo[q] + (int64_t)t * F);
            } else if (a.ibk) {
                if (n <= kIbkK) {
                    double sum = 0.0;
                    for (int i = 0; i < n; ++i) sum += S.yl[j][i];
                    pred[j] = sum / (double)n;
                } else {
                    pred[j] = ibk_nearest_mean_n(n, Kt, S.pu[j], S.yl[j]);
                }
            } else {
                const double* cf = a.coef + ((int64_t)q * RS_NOPT + j) * kTrCoef;
                double yh = cf[0];
                if (n > 1)
                    for (int i = 0; i < n; ++i) yh = fma(cf[1 + i], __ldg(Kt + S.pu[j][i]), yh);
                pred[j] = yh;
            }
        }
        // rank_row's candidates are the optimizations outside the version-mask field: put the
        // excluded ones there (t's own unless all six are ranked, and those outside opt_mask);
        // the fits that are not OK go in the empty-fit field
        const int mfield = ((a.rank_all ? 0 : mt) | ~a.opt_mask) & 63;
        const unsigned long long info64 = (unsigned long long)info | ((unsigned long long)mfield << 30) |
                                          ((unsigned long long)(~okm & 63) << 36);
        rank_row(a.r, rb + t, info64, pred, c);
    }
    if (tid < RS_NOPT) {
        const int st = S.st[tid];
        if (a.fit_status) a.fit_status[(int64_t)q * RS_NOPT + tid] = (uint8_t)st;
        if (a.r.counters && st >= 0 && st <= RS_FIT_NONFINITE) atomicAdd(a.r.counters + 9 + st, 1ull);
    }
    if (a.r.counters) {
        const uint32_t vals[10] = {c.rows, c.pred, c.scored, c.sign, c.rec, c.reck, c.rech, c.t1, c.t1h, c.inv};
        const int slot[10] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 13};
#pragma unroll
        for (int i = 0; i < 10; ++i) {
            const uint32_t v = __reduce_add_sync(0xffffffffu, vals[i]);
            if ((tid & 31) == 0 && v) atomicAdd(a.r.counters + slot[i], (unsigned long long)v);
        }
    }
}

__global__ void iota64_kernel(int64_t* out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = i;
}

}  // namespace

cudaError_t rs_launch_iota64(int64_t* out, int64_t n, cudaStream_t st) {
    if (n > 0) iota64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n);
    return cudaGetLastError();
}

size_t rs_m5p_tree_bytes() { return sizeof(M5Tree); }
int rs_m5p_max_feat() { return kM5MaxFeat; }

size_t rs_transfer_fit_bytes(int64_t Q) {
    return (size_t)Q * RS_NOPT * kTrCoef * sizeof(double) + (size_t)Q * RS_NOPT;
}

cudaError_t rs_launch_transfer(const rs_transfer_args& t, cudaStream_t st) {
    TransferArgs a{};
    a.group_off = t.group_off;
    a.max_runs = t.max_runs;
    a.stat_stride = t.stat_stride;
    a.n_runs = t.n_runs;
    a.a_row = t.a_row_offsets;
    a.a_fw = t.a_feat_width;
    a.a_masks = t.a_masks;
    a.a_lt = t.a_log_time;
    a.b_row = t.b_row_offsets;
    a.b_fw = t.b_feat_width;
    a.b_masks = t.b_masks;
    a.b_lt = t.b_log_time;
    a.KA = t.KA;
    a.Kx = t.Kx;
    a.ld = t.ld;
    a.lambda = t.lambda;
    a.coef = t.fit_ws;
    a.fst = reinterpret_cast<uint8_t*>(t.fit_ws + (size_t)t.Q * RS_NOPT * kTrCoef);
    a.ibk = t.ibk;
    a.opt_mask = t.opt_mask & 63;
    a.rank_all = (t.flags & RS_RANK_ALL) != 0;
    a.fit_status = t.fit_status;
    a.m5p = t.m5p;
    a.trees = reinterpret_cast<M5Tree*>(t.m5_ws);
    a.ZA = t.ZA;
    a.a_xo = t.a_x_offsets;
    a.ZB = t.ZB;
    a.b_xo = t.b_x_offsets;
    a.r = RankPassArgs{nullptr, 0, nullptr, 0, 0, nullptr, t.dstatus, t.k, okey_host(t.log_tau),
                       t.flags & ~RS_RANK_ALL, t.rec_code, t.rec_pred, t.pred_all, t.counters};
    cudaError_t e = cudaSuccess;
    if (t.m5p) {
        const size_t msmem = sizeof(M5Smem);
        e = cudaFuncSetAttribute(m5p_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem);
        if (e != cudaSuccess) return e;
        m5p_fit_kernel<<<dim3((unsigned)t.Q, RS_NOPT), kM5Threads, msmem, st>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    } else if (!t.ibk) {
        const int nmax = RS_MAXPAIRS * t.max_runs;
        const size_t fsmem = ((size_t)nmax * (nmax + 1) + 5 * (size_t)nmax) * sizeof(double);
        e = cudaFuncSetAttribute(transfer_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
        if (e != cudaSuccess) return e;
        transfer_fit_kernel<<<dim3((unsigned)t.Q, RS_NOPT), kTrThreads, fsmem, st>>>(a, nmax);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const size_t smem = sizeof(RankSmem);
    e = cudaFuncSetAttribute(transfer_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    transfer_rank_kernel<<<(unsigned)t.Q, RS_MAXV, smem, st>>>(a);
    return cudaGetLastError();
}
