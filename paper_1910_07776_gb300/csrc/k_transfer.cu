// Table 2 transfer (Sec. 5): the fits of each problem's training group of runs (one block per
// problem and optimization), then the predictions for its test program, ranking and scoring
// (one block per problem).
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
            if (a.ibk) {
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
    a.r = RankPassArgs{nullptr, 0, nullptr, 0, 0, nullptr, t.dstatus, t.k, okey_host(t.log_tau),
                       t.flags & ~RS_RANK_ALL, t.rec_code, t.rec_pred, t.pred_all, t.counters};
    cudaError_t e = cudaSuccess;
    if (!t.ibk) {
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
