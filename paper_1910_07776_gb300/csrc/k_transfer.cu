// Table 2 transfer (Sec. 5): the fits of each problem's training group of runs, the
// predictions for its test program, ranking and scoring -- one block per problem.
#include "rank_row.cuh"

namespace {

// ====================================================================== transfer (Table 2)
// One block per transfer problem q: the fits of its training group (every before/after pair
// of every run, run by run in ascending before slot, a pair never spanning two runs), the
// predictions for every version t of its test program, ranking and scoring.  The group's
// versions form one list of N (rs_group_layout); KA[q] is their Gram, Kx[q][t][u] the block
// between test row t and version u (dot products; squared distances for IBK).
// Ridge: the bordered dual system of each optimization, M = KA(pairs) + lambda I = L D L^T
// (right-looking, one thread per row, in shared memory), then b and alpha as in fit_fixed and
// the prediction b + sum_a alpha_a Kx[t][u_a].  IBK: the mean label of the kIbkK pairs
// nearest to t.  Candidates: outside t's mask (all six with RS_RANK_ALL) and inside
// opt_mask; ranking, threshold, top-k and scoring as in the rank pass with the test
// program's own times.
constexpr int kTrPairs = RS_MAXPAIRS * RS_MAXRUNS;   // pairs of one fit
constexpr int kTrRows = RS_MAXV * RS_MAXRUNS;        // versions of one group
constexpr int kTrThreads = kTrPairs;                 // one thread per matrix row
constexpr int kTrLd = kTrPairs + 1;

struct TransferSmem {
    double M[kTrPairs * kTrLd];          // the factor (lower triangle, D on the diagonal)
    double col[kTrPairs];
    double ty[kTrPairs], t1[kTrPairs];
    double coef[RS_NOPT][kTrPairs + 1];  // b, alpha
    double yl[RS_NOPT][kTrPairs];
    double lt_a[kTrRows];
    double lt_b[RS_MAXV];
    double bval;
    uint16_t pu[RS_NOPT][kTrPairs];      // group version of each pair's before side
    uint8_t msk_a[kTrRows];
    int8_t slot_a[RS_MAXRUNS][RS_MAXV];
    uint8_t msk_b[RS_MAXV];
    int8_t slot_b[RS_MAXV];
    int np[RS_NOPT], st[RS_NOPT];
};

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
    int ibk, opt_mask, rank_all;
    uint8_t* fit_status;
    RankPassArgs r;                      // k, ktau, flags (without RS_RANK_ALL), outputs, counters
};

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

// The bordered ridge system of one fit with n >= 2 pairs, block-wide.  Writes b, alpha into
// coef and returns the status (the same for every thread).
__device__ int transfer_fit(TransferSmem& S, int j, int n, const double* __restrict__ KAq, int ld, double lambda) {
    const int tid = threadIdx.x;
    for (int e = tid; e < n * n; e += kTrThreads) {
        const int i = e / n, c = e - i * n;
        if (c <= i) S.M[i * kTrLd + c] = __ldg(KAq + (int64_t)S.pu[j][i] * ld + S.pu[j][c]) + (i == c ? lambda : 0.0);
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const double d = S.M[k * kTrLd + k];
        if (!pos_finite(d)) return RS_FIT_NOTPD;      // every thread read the same pivot
        const double dinv = 1.0 / d;
        if (tid > k && tid < n) S.col[tid] = S.M[tid * kTrLd + k];
        __syncthreads();
        if (tid > k && tid < n) {
            const double l = S.col[tid] * dinv;
            for (int c = k + 1; c <= tid; ++c) S.M[tid * kTrLd + c] = fma(-l, S.col[c], S.M[tid * kTrLd + c]);
            S.M[tid * kTrLd + k] = l;
        }
        __syncthreads();
    }
    if (tid < n) {                               // L t = rhs, two right-hand sides
        S.ty[tid] = S.yl[j][tid];
        S.t1[tid] = 1.0;
    }
    __syncthreads();
    for (int k = 0; k < n - 1; ++k) {
        if (tid > k && tid < n) {
            const double l = S.M[tid * kTrLd + k];
            S.ty[tid] = fma(-l, S.ty[k], S.ty[tid]);
            S.t1[tid] = fma(-l, S.t1[k], S.t1[tid]);
        }
        __syncthreads();
    }
    if (tid == 0) {
        double num = 0.0, den = 0.0;
        for (int i = 0; i < n; ++i) {
            const double sc = S.t1[i] / S.M[i * kTrLd + i];
            num = fma(sc, S.ty[i], num);
            den = fma(sc, S.t1[i], den);
        }
        S.bval = num / den;
    }
    __syncthreads();
    const double b = S.bval;
    if (tid < n) S.ty[tid] = fma(-b, S.t1[tid], S.ty[tid]) / S.M[tid * kTrLd + tid];
    __syncthreads();
    for (int k = n - 1; k > 0; --k) {            // L^T alpha = D^-1 (t_y - b t_1)
        if (tid < k) S.ty[tid] = fma(-S.M[k * kTrLd + tid], S.ty[k], S.ty[tid]);
        __syncthreads();
    }
    bool fin = finite_bits(b);
    if (tid < n) {
        S.coef[j][1 + tid] = S.ty[tid];
        fin = finite_bits(S.ty[tid]);
    }
    if (tid == 0) S.coef[j][0] = b;
    return __syncthreads_and(fin || tid >= n) && finite_bits(b) ? RS_FIT_OK : RS_FIT_NONFINITE;
}

__global__ void __launch_bounds__(kTrThreads, 1)
transfer_kernel(const TransferArgs a) {
    extern __shared__ __align__(16) unsigned char tsm[];
    TransferSmem& S = *reinterpret_cast<TransferSmem*>(tsm);
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
    for (int e = tid; e < RS_MAXRUNS * RS_MAXV; e += kTrThreads) S.slot_a[e / RS_MAXV][e % RS_MAXV] = -1;
    if (tid < RS_MAXV) S.slot_b[tid] = -1;
    for (int u = tid; u < N; u += kTrThreads) {
        int r = 0;
        while (u >= start[r + 1]) ++r;
        const int64_t row = a.a_row[g0 + r] + (u - start[r]);
        S.msk_a[u] = a.a_masks[row] & 63;
        S.lt_a[u] = a.a_lt[row];
    }
    if (tid < VB) {
        S.msk_b[tid] = a.b_masks[rb + tid] & 63;
        S.lt_b[tid] = a.b_lt[rb + tid];
    }
    __syncthreads();
    for (int u = tid; u < N; u += kTrThreads) {
        int r = 0;
        while (u >= start[r + 1]) ++r;
        S.slot_a[r][S.msk_a[u]] = (int8_t)(u - start[r]);
    }
    if (tid < VB) S.slot_b[S.msk_b[tid]] = (int8_t)tid;
    __syncthreads();
    if (tid < RS_NOPT) {
        const int j = tid;
        int np = 0;
        for (int r = 0; r < R; ++r)
            for (int u = start[r]; u < start[r + 1]; ++u) {
                const int m = S.msk_a[u];
                if ((m >> j) & 1) continue;
                const int w = S.slot_a[r][m | (1 << j)];
                if (w < 0) continue;
                if (np == kTrPairs) {            // only possible with repeated masks
                    rs_dev_flag(a.r.dstatus, RS_EDATA, q);
                    continue;
                }
                S.pu[j][np] = (uint16_t)u;
                S.yl[j][np] = S.lt_a[u] - S.lt_a[start[r] + w];
                ++np;
            }
        S.np[j] = np;
        S.st[j] = np > 0 ? RS_FIT_OK : RS_FIT_EMPTY;
        if (np == 1) {                           // one pair: alpha = 0, b = its label
            S.coef[j][0] = S.yl[j][0];
            S.coef[j][1] = 0.0;
            if (!finite_bits(S.yl[j][0])) S.st[j] = RS_FIT_NONFINITE;
        }
    }
    __syncthreads();
    if (!a.ibk) {
        const double* KAq = a.KA + (int64_t)q * a.ld * a.ld;
        for (int j = 0; j < RS_NOPT; ++j) {
            const int n = S.np[j];
            if (n < 2) continue;
            const int st = transfer_fit(S, j, n, KAq, a.ld, a.lambda);
            __syncthreads();
            if (tid == 0) S.st[j] = st;
        }
        __syncthreads();
    }
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
            if (a.ibk) {
                if (n <= kIbkK) {
                    double sum = 0.0;
                    for (int i = 0; i < n; ++i) sum += S.yl[j][i];
                    pred[j] = sum / (double)n;
                } else {
                    pred[j] = ibk_nearest_mean_n(n, Kt, S.pu[j], S.yl[j]);
                }
            } else {
                double yh = S.coef[j][0];
                if (n > 1)
                    for (int i = 0; i < n; ++i) yh = fma(S.coef[j][1 + i], __ldg(Kt + S.pu[j][i]), yh);
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
        if (a.r.counters) atomicAdd(a.r.counters + 9 + st, 1ull);
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
    a.ibk = t.ibk;
    a.opt_mask = t.opt_mask & 63;
    a.rank_all = (t.flags & RS_RANK_ALL) != 0;
    a.fit_status = t.fit_status;
    a.r = RankPassArgs{nullptr, 0, nullptr, 0, 0, nullptr, t.dstatus, t.k, okey_host(t.log_tau),
                       t.flags & ~RS_RANK_ALL, t.rec_code, t.rec_pred, t.pred_all, t.counters};
    const size_t smem = sizeof(TransferSmem);
    cudaError_t e = cudaFuncSetAttribute(transfer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    transfer_kernel<<<(unsigned)t.Q, kTrThreads, smem, st>>>(a);
    return cudaGetLastError();
}
