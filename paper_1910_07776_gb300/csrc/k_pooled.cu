// k_pooled.cu -- pooled ridge fits in primal form (A3 + A4): one model per optimization j
// trained on the before/after pairs (Sec. 3.3) of MANY programs at once, the training set of a
// tool that has seen many codes (Sec. 5's transfer between codes, at scale).  With n pairs
// far more numerous than the F features, the primal normal equations are the small system:
//     G_j = sum_a c_a c_a^T + lambda I,   r_j = sum_a c_a (y_a - ybar_j),   c_a = z_a - zbar_j,
//     G_j beta_j = r_j,   b_j = ybar_j - zbar_j . beta_j      (the intercept unpenalised).
// The Gram X^T W X (W selecting the pairs of optimization j, centred) is the dense contraction:
// it runs on the tcgen05 tensor cores as one batched GEMM over j, with the BF16 hi/lo split of
// the centred rows (c = hi + lo; G ~ hi hi^T + hi lo^T + lo hi^T, K = 3 n), the operands
// staged feature-major by a transpose kernel and fed by TMA.  The FP64 Cholesky factorisation
// of G_j follows, and (RS_REFINE_X) one step of iterative refinement whose residual
// r_j - lambda beta - sum_a c_a (c_a . beta) is taken exactly in FP64 through the rows.
// Predictions: b_j + z_t . beta_j for every version t of a batch, ranked and scored by
// rank_row (Sec. 2 tier 3).
#include "rank_row.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int kPoolMaxPairs = 65536;   // pairs per optimization (all programs together)
constexpr int kSolveThreads = 512;

struct PoolArgs {
    int P, F;
    const int64_t* row_off;
    const int32_t* fw;
    const int64_t* x_off;
    const double* Z;
    const uint8_t* masks;
    const double* lt;
    const uint8_t* use;          // nullable: programs that train
    int* counts;                 // [6][P]
    int64_t* offs;               // [6][P + 1]
    int64_t* zoff;               // [6][NP]: offset in Z of the before version's features
    double* y;                   // [6][NP]: log speedup of the pair
    int NP;                      // pairs capacity per optimization
    double* zbar;                // [6][F]
    double* ybar;                // [6]
    double* G;                   // [6][F][F]
    double* r;                   // [6][F]
    double* rho;                 // [6][F]
    double* s;                   // [6][NP]: c_a . beta during refinement
    double* coef;                // [6][F + 1]: b, beta
    uint8_t* status;             // [6]
    double lambda;
    int* dstatus;
};

// Per program (block of 64 threads, thread = version slot): the number of pairs of each j.
__global__ void __launch_bounds__(RS_MAXV) pooled_count_kernel(PoolArgs a) {
    __shared__ int8_t slot_of[64];
    __shared__ int cnt[RS_NOPT];
    const int p = blockIdx.x, v = threadIdx.x;
    const int64_t r0 = a.row_off[p];
    const int V = (int)(a.row_off[p + 1] - r0);
    slot_of[v] = -1;
    if (v < RS_NOPT) cnt[v] = 0;
    __syncthreads();
    const bool want = !a.use || a.use[p];
    const bool valid = V >= 1 && V <= RS_MAXV && a.fw[p] == a.F;
    if (want && !valid && v == 0) rs_dev_flag(a.dstatus, RS_EDATA, p);   // skipped, reported
    const bool use = want && valid;
    const int m = use && v < V ? (a.masks[r0 + v] & 63) : 0;
    if (use && v < V) slot_of[m] = (int8_t)v;
    __syncthreads();
    if (use && v < V)
        for (int j = 0; j < RS_NOPT; ++j)
            if (!((m >> j) & 1) && slot_of[m | (1 << j)] >= 0) atomicAdd(&cnt[j], 1);
    __syncthreads();
    if (v < RS_NOPT) a.counts[v * a.P + p] = use ? cnt[v] : 0;
}

// Per j (one block): exclusive prefix of the per-program counts.
__global__ void __launch_bounds__(1024) pooled_scan_kernel(PoolArgs a) {
    __shared__ long long wsum[32];
    const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int chunk = (a.P + 1023) / 1024;
    const int p0 = tid * chunk, p1 = p0 + chunk < a.P ? p0 + chunk : a.P;
    long long s = 0;
    for (int p = p0; p < p1; ++p) s += a.counts[j * a.P + p];
    long long incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long w = wsum[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    long long off = incl - s + (warp > 0 ? wsum[warp - 1] : 0ll);
    int64_t* o = a.offs + (int64_t)j * (a.P + 1);
    for (int p = p0; p < p1; ++p) {
        o[p] = off;
        off += a.counts[j * a.P + p];
    }
    if (tid == 1023) o[a.P] = off;
}

// Per program: its pairs of each j, in ascending order of the before slot, after the pairs of
// the programs before it.
__global__ void __launch_bounds__(RS_MAXV) pooled_fill_kernel(PoolArgs a) {
    __shared__ int8_t slot_of[64];
    __shared__ int wcnt[RS_NOPT][2];
    const int p = blockIdx.x, v = threadIdx.x, lane = v & 31, warp = v >> 5;
    const int64_t r0 = a.row_off[p];
    const int V = (int)(a.row_off[p + 1] - r0);
    const bool use = (!a.use || a.use[p]) && V >= 1 && V <= RS_MAXV && a.fw[p] == a.F;
    slot_of[v] = -1;
    __syncthreads();
    const int m = v < V ? (a.masks[r0 + v] & 63) : 0;
    if (use && v < V) slot_of[m] = (int8_t)v;
    __syncthreads();
    for (int j = 0; j < RS_NOPT; ++j) {
        const int w = (use && v < V && !((m >> j) & 1)) ? slot_of[m | (1 << j)] : -1;
        const unsigned bal = __ballot_sync(0xffffffffu, w >= 0);
        if (lane == 0) wcnt[j][warp] = __popc(bal);
        __syncthreads();
        if (w >= 0) {
            const int64_t pos = a.offs[(int64_t)j * (a.P + 1) + p] + (warp ? wcnt[j][0] : 0) +
                                __popc(bal & ((1u << lane) - 1u));
            if (pos < a.NP) {
                a.zoff[(int64_t)j * a.NP + pos] = a.x_off[p] + (int64_t)v * a.F;
                a.y[(int64_t)j * a.NP + pos] = a.lt[r0 + v] - a.lt[r0 + w];
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int n_pairs(const PoolArgs& a, int j) {
    const int64_t n = a.offs[(int64_t)j * (a.P + 1) + a.P];
    return (int)(n < a.NP ? n : a.NP);
}
__device__ __forceinline__ const double* zrow(const PoolArgs& a, int64_t zo) { return a.Z + zo; }

// Means of the pairs' features and labels, per j; thread f sums over the pairs in order.
__global__ void __launch_bounds__(128) pooled_mean_kernel(PoolArgs a) {
    const int j = blockIdx.y, f = blockIdx.x * 128 + threadIdx.x;
    const int n = n_pairs(a, j);
    const int64_t* rows = a.zoff + (int64_t)j * a.NP;
    if (f < a.F) {
        double s = 0.0;
        for (int q = 0; q < n; ++q) s += __ldg(zrow(a, rows[q]) + f);
        a.zbar[j * a.F + f] = n > 0 ? s / n : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < n; ++q) s += a.y[(int64_t)j * a.NP + q];
        a.ybar[j] = n > 0 ? s / n : 0.0;
    }
}

// The GEMM operands: A_j = [hi | hi | lo], B_j = [hi | lo | hi] of the centred rows, stored
// feature-major ([6][F][3 Np], pair index contiguous, zero past n_j).  Block (tile of 64 pairs,
// j): the tile's centred values in shared memory, 32 features at a time, written transposed.
__global__ void __launch_bounds__(256)
pooled_stage_kernel(PoolArgs a, int Np, __nv_bfloat16* A, __nv_bfloat16* B) {
    __shared__ double t[64][33];
    const int j = blockIdx.y, k0 = blockIdx.x * 64;
    const int n = n_pairs(a, j);
    const int64_t* rows = a.zoff + (int64_t)j * a.NP;
    const double* zb = a.zbar + j * a.F;
    for (int f0 = 0; f0 < a.F; f0 += 32) {
        for (int e = threadIdx.x; e < 64 * 32; e += 256) {        // read: pairs x features
            const int q = e >> 5, f = f0 + (e & 31);
            double c = 0.0;
            if (k0 + q < n && f < a.F) c = __ldg(zrow(a, rows[k0 + q]) + f) - zb[f];
            t[q][e & 31] = c;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * 64; e += 256) {        // write: features x pairs
            const int fl = e >> 6, q = e & 63, f = f0 + fl;
            if (f < a.F) {
                const float cf = (float)t[q][fl];
                const __nv_bfloat16 hi = __float2bfloat16(cf);
                const __nv_bfloat16 lo = __float2bfloat16(cf - __bfloat162float(hi));
                const int64_t base = ((int64_t)j * a.F + f) * 3 * Np + k0 + q;
                A[base] = hi;
                A[base + Np] = hi;
                A[base + 2 * Np] = lo;
                B[base] = hi;
                B[base + Np] = lo;
                B[base + 2 * Np] = hi;
            }
        }
        __syncthreads();
    }
}

struct EpiPooled {
    double* G;
    int F;
    __device__ void operator()(int z, int row, int col0, const float (&v)[16]) const {
        double* g = G + ((int64_t)z * F + row) * F;
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (col0 + i < F) g[col0 + i] = (double)v[i];
    }
};

// r_j[f] = sum_a c_a[f] (y_a - ybar_j), in pair order (FP64, exact centring).
__global__ void __launch_bounds__(128) pooled_rhs_kernel(PoolArgs a) {
    const int j = blockIdx.y, f = blockIdx.x * 128 + threadIdx.x;
    if (f >= a.F) return;
    const int n = n_pairs(a, j);
    const int64_t* rows = a.zoff + (int64_t)j * a.NP;
    const double zb = a.zbar[j * a.F + f], yb = a.ybar[j];
    double s = 0.0;
    for (int q = 0; q < n; ++q) s = fma(__ldg(zrow(a, rows[q]) + f) - zb, a.y[(int64_t)j * a.NP + q] - yb, s);
    a.r[j * a.F + f] = s;
}

// Per j (one block): Cholesky G + lambda I = L L^T in place (right-looking, the trailing
// update spread over the block), then L L^T beta = r.  With refine = 1 the factor is already
// there: only the solve, of the residual, added to beta.
__global__ void __launch_bounds__(kSolveThreads) pooled_solve_kernel(PoolArgs a, int refine) {
    __shared__ double col[512];
    __shared__ int bad;
    const int j = blockIdx.x, F = a.F, tid = threadIdx.x;
    double* G = a.G + (int64_t)j * F * F;
    const int n = n_pairs(a, j);
    if (tid == 0) bad = 0;
    __syncthreads();
    if (n == 0) {
        if (tid == 0 && !refine) {
            a.status[j] = RS_FIT_EMPTY;
            a.coef[(int64_t)j * (F + 1)] = nan_d();
        }
        return;
    }
    if (!refine) {
        for (int i = tid; i < F; i += kSolveThreads) G[(int64_t)i * F + i] += a.lambda;
        __syncthreads();
        for (int k = 0; k < F; ++k) {
            const double d = G[(int64_t)k * F + k];
            if (!(d > 0.0) || !isfinite(d)) {
                if (tid == 0) bad = 1;
                break;
            }
            const double l = sqrt(d);
            const double il = 1.0 / l;
            for (int i = k + 1 + tid; i < F; i += kSolveThreads) {
                const double v = G[(int64_t)i * F + k] * il;
                G[(int64_t)i * F + k] = v;
                col[i] = v;
            }
            __syncthreads();
            if (tid == 0) G[(int64_t)k * F + k] = l;
            const int m = F - k - 1;
            for (int e = tid; e < m * m; e += kSolveThreads) {          // lower part of the square
                const int i = k + 1 + e / m, c = k + 1 + e % m;
                if (c <= i) G[(int64_t)i * F + c] = fma(-col[i], col[c], G[(int64_t)i * F + c]);
            }
            __syncthreads();
        }
        __syncthreads();
        if (bad) {
            if (tid == 0) {
                a.status[j] = RS_FIT_NOTPD;
                a.coef[(int64_t)j * (F + 1)] = nan_d();
            }
            return;
        }
    } else if (a.status[j] != RS_FIT_OK) {
        return;
    }
    // L L^T x = rhs: rhs = r (first solve) or the residual rho (refinement); x in col[]
    const double* rhs = refine ? a.rho + j * F : a.r + j * F;
    for (int i = tid; i < F; i += kSolveThreads) col[i] = rhs[i];
    __syncthreads();
    for (int k = 0; k < F; ++k) {                                     // forward
        if (tid == 0) col[k] /= G[(int64_t)k * F + k];
        __syncthreads();
        for (int i = k + 1 + tid; i < F; i += kSolveThreads) col[i] = fma(-G[(int64_t)i * F + k], col[k], col[i]);
        __syncthreads();
    }
    for (int k = F - 1; k >= 0; --k) {                                // backward
        if (tid == 0) col[k] /= G[(int64_t)k * F + k];
        __syncthreads();
        for (int i = tid; i < k; i += kSolveThreads) col[i] = fma(-G[(int64_t)k * F + i], col[k], col[i]);
        __syncthreads();
    }
    double* beta = a.coef + (int64_t)j * (F + 1) + 1;
    for (int i = tid; i < F; i += kSolveThreads) beta[i] = refine ? beta[i] + col[i] : col[i];
    __syncthreads();
    if (tid == 0) {
        double b = a.ybar[j];
        bool fin = true;
        for (int f = 0; f < F; ++f) {
            b = fma(-a.zbar[j * F + f], beta[f], b);
            fin = fin && isfinite(beta[f]);
        }
        a.coef[(int64_t)j * (F + 1)] = b;
        a.status[j] = (fin && isfinite(b)) ? RS_FIT_OK : RS_FIT_NONFINITE;
    }
}

// Refinement, step 1: s_a = c_a . beta_j for every pair (one warp per pair).
__global__ void __launch_bounds__(256) pooled_project_kernel(PoolArgs a) {
    const int j = blockIdx.y;
    const int q = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int n = n_pairs(a, j);
    if (q >= n) return;
    const double* z = zrow(a, a.zoff[(int64_t)j * a.NP + q]);
    const double* zb = a.zbar + j * a.F;
    const double* beta = a.coef + (int64_t)j * (a.F + 1) + 1;
    double s = 0.0;
    for (int f = lane; f < a.F; f += 32) s = fma(__ldg(z + f) - zb[f], beta[f], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) a.s[(int64_t)j * a.NP + q] = s;
}

// Refinement, step 2: rho_j[f] = r_j[f] - lambda beta_j[f] - sum_a c_a[f] s_a (pair order).
__global__ void __launch_bounds__(128) pooled_residual_kernel(PoolArgs a) {
    const int j = blockIdx.y, f = blockIdx.x * 128 + threadIdx.x;
    if (f >= a.F) return;
    const int n = n_pairs(a, j);
    const int64_t* rows = a.zoff + (int64_t)j * a.NP;
    const double zb = a.zbar[j * a.F + f];
    double acc = 0.0;
    for (int q = 0; q < n; ++q) acc = fma(__ldg(zrow(a, rows[q]) + f) - zb, a.s[(int64_t)j * a.NP + q], acc);
    const double beta = a.coef[(int64_t)j * (a.F + 1) + 1 + f];
    a.rho[j * a.F + f] = a.r[j * a.F + f] - a.lambda * beta - acc;
}

// Predictions of the pooled models for every version of a batch (one block per program,
// thread = version slot), ranked and scored against the program's own times.
struct PoolPredArgs {
    int F;
    const int64_t* row_off;
    const int32_t* fw;
    const int64_t* x_off;
    const double* Z;
    const uint8_t* masks;
    const double* lt;
    const double* coef;       // [6][F + 1]
    const uint8_t* status;    // [6]
    int rank_all;
    RankPassArgs r;
};

__global__ void __launch_bounds__(RS_MAXV) pooled_predict_kernel(PoolPredArgs a) {
    __shared__ double lt_s[RS_MAXV];
    __shared__ uint8_t msk_s[RS_MAXV];
    __shared__ int8_t slot_s[RS_MAXV];
    const int p = blockIdx.x, t = threadIdx.x;
    const int64_t r0 = a.row_off[p];
    const int V = (int)(a.row_off[p + 1] - r0);
    const bool okp = V >= 1 && V <= RS_MAXV && a.fw[p] == a.F;
    if (!okp) {
        if (t == 0) rs_dev_flag(a.r.dstatus, RS_EDATA, p);
        return;
    }
    slot_s[t] = -1;
    if (t < V) {
        msk_s[t] = a.masks[r0 + t] & 63;
        lt_s[t] = a.lt[r0 + t];
    }
    __syncthreads();
    if (t < V) slot_s[msk_s[t]] = (int8_t)t;
    __syncthreads();
    RankTally c;
    if (t < V) {
        const int mt = msk_s[t];
        const uint32_t info = row_summary(t, V, msk_s, lt_s, slot_s);
        int okm = 0;
#pragma unroll
        for (int j = 0; j < RS_NOPT; ++j) okm |= (a.status[j] == RS_FIT_OK) << j;
        const int candm = (a.rank_all ? 63 : (~mt & 63)) & okm;
        const double* z = a.Z + a.x_off[p] + (int64_t)t * a.F;
        double pred[RS_NOPT];
#pragma unroll
        for (int j = 0; j < RS_NOPT; ++j) {
            pred[j] = 0.0;
            if (!((candm >> j) & 1)) continue;
            const double* cf = a.coef + (int64_t)j * (a.F + 1);
            double yh = cf[0];
            for (int f = 0; f < a.F; ++f) yh = fma(__ldg(z + f), cf[1 + f], yh);
            pred[j] = yh;
        }
        const int mfield = a.rank_all ? 0 : mt;
        const unsigned long long info64 = (unsigned long long)info | ((unsigned long long)mfield << 30) |
                                          ((unsigned long long)(~okm & 63) << 36);
        rank_row(a.r, r0 + t, info64, pred, c);
    }
    if (a.r.counters) {
        const uint32_t vals[10] = {c.rows, c.pred, c.scored, c.sign, c.rec, c.reck, c.rech, c.t1, c.t1h, c.inv};
        const int slot[10] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 13};
#pragma unroll
        for (int i = 0; i < 10; ++i) {
            const uint32_t v = __reduce_add_sync(0xffffffffu, vals[i]);
            if ((t & 31) == 0 && v) atomicAdd(a.r.counters + slot[i], (unsigned long long)v);
        }
    }
}

int pairs_cap(int64_t P) {
    const int64_t np = P * 32;
    return (int)(np < kPoolMaxPairs ? np : kPoolMaxPairs);
}
int padded_pairs(int64_t P) { return (pairs_cap(P) + 63) / 64 * 64; }

struct PoolWs {
    int* counts;
    int64_t* offs;
    int64_t* zoff;
    double *y, *zbar, *ybar, *G, *r, *rho, *s;
    __nv_bfloat16 *A, *B;
    size_t bytes;
};

PoolWs carve_pool(void* base, int64_t P, int F) {
    PoolWs w{};
    char* c = (char*)base;
    size_t o = 0;
    auto take = [&](size_t n) -> void* {
        void* p = c ? (void*)(c + o) : nullptr;
        o += (n + 255) & ~(size_t)255;
        return p;
    };
    const int NP = pairs_cap(P), Np = padded_pairs(P);
    w.counts = (int*)take((size_t)RS_NOPT * P * sizeof(int));
    w.offs = (int64_t*)take((size_t)RS_NOPT * (P + 1) * sizeof(int64_t));
    w.zoff = (int64_t*)take((size_t)RS_NOPT * NP * sizeof(int64_t));
    w.y = (double*)take((size_t)RS_NOPT * NP * sizeof(double));
    w.s = (double*)take((size_t)RS_NOPT * NP * sizeof(double));
    w.zbar = (double*)take((size_t)RS_NOPT * F * sizeof(double));
    w.ybar = (double*)take(RS_NOPT * sizeof(double));
    w.G = (double*)take((size_t)RS_NOPT * F * F * sizeof(double));
    w.r = (double*)take((size_t)RS_NOPT * F * sizeof(double));
    w.rho = (double*)take((size_t)RS_NOPT * F * sizeof(double));
    w.A = (__nv_bfloat16*)take((size_t)RS_NOPT * F * 3 * Np * sizeof(__nv_bfloat16));
    w.B = (__nv_bfloat16*)take((size_t)RS_NOPT * F * 3 * Np * sizeof(__nv_bfloat16));
    w.bytes = o;
    return w;
}

}  // namespace

size_t rs_pooled_workspace_bytes_impl(int64_t P, int F) { return carve_pool(nullptr, P, F).bytes; }

cudaError_t rs_launch_fit_pooled(const rs_batch* b, const uint8_t* use, double lambda, int refine, void* ws,
                                 size_t ws_bytes, double* coef, uint8_t* status, int* dstatus, cudaStream_t st) {
    const int64_t P = b->n_programs;
    const int F = b->max_feat;
    PoolWs w = carve_pool(ws, P, F);
    if (!ws || ws_bytes < w.bytes || F > 512 || P > 65535) return cudaErrorInvalidValue;
    PoolArgs a{};
    a.P = (int)P;
    a.F = F;
    a.row_off = b->row_offsets;
    a.fw = b->feat_width;
    a.x_off = b->x_offsets;
    a.Z = (const double*)b->X;
    a.masks = b->masks;
    a.lt = b->log_time;
    a.use = use;
    a.counts = w.counts;
    a.offs = w.offs;
    a.zoff = w.zoff;
    a.y = w.y;
    a.NP = pairs_cap(P);
    a.zbar = w.zbar;
    a.ybar = w.ybar;
    a.G = w.G;
    a.r = w.r;
    a.rho = w.rho;
    a.s = w.s;
    a.coef = coef;
    a.status = status;
    a.lambda = lambda;
    a.dstatus = dstatus;
    const int Np = padded_pairs(P);
    const unsigned fb = (unsigned)((F + 127) / 128);
    pooled_count_kernel<<<(unsigned)P, RS_MAXV, 0, st>>>(a);
    pooled_scan_kernel<<<RS_NOPT, 1024, 0, st>>>(a);
    pooled_fill_kernel<<<(unsigned)P, RS_MAXV, 0, st>>>(a);
    pooled_mean_kernel<<<dim3(fb, RS_NOPT), 128, 0, st>>>(a);
    pooled_stage_kernel<<<dim3((unsigned)(Np / 64), RS_NOPT), 256, 0, st>>>(a, Np, w.A, w.B);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CUtensorMap ta, tb;
    e = rs_make_tmap_bf16_3d(&ta, w.A, RS_NOPT, F, 3 * Np, 3 * Np, tc::BM);
    if (e == cudaSuccess) e = rs_make_tmap_bf16_3d(&tb, w.B, RS_NOPT, F, 3 * Np, 3 * Np, 64);
    if (e == cudaSuccess)
        e = tc::gemm_launch<64, 4, EpiPooled, true>(ta, tb, F, F, 3 * Np, RS_NOPT, EpiPooled{w.G, F}, dstatus, st);
    if (e != cudaSuccess) return e;
    pooled_rhs_kernel<<<dim3(fb, RS_NOPT), 128, 0, st>>>(a);
    pooled_solve_kernel<<<RS_NOPT, kSolveThreads, 0, st>>>(a, 0);
    if (refine) {
        pooled_project_kernel<<<dim3((unsigned)((a.NP + 7) / 8), RS_NOPT), 256, 0, st>>>(a);
        pooled_residual_kernel<<<dim3(fb, RS_NOPT), 128, 0, st>>>(a);
        pooled_solve_kernel<<<RS_NOPT, kSolveThreads, 0, st>>>(a, 1);
    }
    return cudaGetLastError();
}

cudaError_t rs_launch_predict_pooled(const rs_batch* b, const double* coef, const uint8_t* status, int k,
                                     double log_tau, int flags, uint32_t* rec_code, double* rec_pred,
                                     double* pred_all, unsigned long long* counters, int* dstatus, cudaStream_t st) {
    PoolPredArgs a{};
    a.F = b->max_feat;
    a.row_off = b->row_offsets;
    a.fw = b->feat_width;
    a.x_off = b->x_offsets;
    a.Z = (const double*)b->X;
    a.masks = b->masks;
    a.lt = b->log_time;
    a.coef = coef;
    a.status = status;
    a.rank_all = (flags & RS_RANK_ALL) ? 1 : 0;
    RankPassArgs& r = a.r;
    r.dstatus = dstatus;
    r.k = k;
    r.ktau = okey_host(log_tau);
    r.flags = 0;                  // candidates come through the version-mask field
    r.rec_code = rec_code;
    r.rec_pred = rec_pred;
    r.pred_all = pred_all;
    r.counters = counters;
    pooled_predict_kernel<<<(unsigned)b->n_programs, RS_MAXV, 0, st>>>(a);
    return cudaGetLastError();
}
