// K3 + K4: batched ridge fits, predictions, ranking and scoring (Sec. 2 tiers 2 and 3,
// Sec. 3.3 pairs, Sec. 3.4 regression family, Sec. 5 protocol, Sec. 6 / Table 3 metric).
//
// Fit (per split s and optimization j): the n training pairs are the pairs (v, v|j) with
// both versions in the train mask (Sec. 3.3); a pair carries the feature vector of v and
// the label log t(v) - log t(v|j) (Sec. 5).  With the per-program Gram block K
// (uncentred), ridge with an unpenalised intercept is the bordered system
//       (K_TT + lambda I) alpha + b 1 = y,      1^T alpha = 0
// (stationarity in beta = sum_a alpha_a z_a and in b).  With M = K_TT + lambda I = L L^T
// (FP64 Cholesky): u = M^-1 y, w = M^-1 1, b = 1^T u / 1^T w, alpha = u - b w.  The
// prediction for a test version t is b + sum_a alpha_a K[t][v_a] (= b + z_t . beta).
//
// This part's FP64 pipe is narrow: one FP64 warp instruction holds an SM sub-partition's
// FP64 unit for many cycles whatever the number of active lanes.  So the batched form
// never lets fits of different sizes share a warp:
//   pairs  -> per program and optimization, the before/after version pairs and labels;
//   plan   -> per fit, the mask of its training pairs and its size n; histogram of n;
//   bucket -> a counting sort of all fits of the batch by n;
//   solve  -> n <= kNReg: one fit per thread, fully unrolled for that n, registers only;
//             kNReg < n <= kNMid: one fit per thread, factor in shared memory;
//             n >  kNMid: one fit per warp, lanes = matrix rows;
//   rank   -> per chunk of splits of one program: predictions, sort, threshold, top-k,
//             scores; comparisons on order-preserving integer keys (no FP64 compares).
// Reciprocal square roots of the pivots come from an FP32 seed refined by two Newton
// steps in FP64 (fewer FP64 instructions than a division and a square root).
// The plain form solves every fit with one warp inside the rank kernel (no bucketing).
#include <math.h>
#include <string.h>

#include "mbar.cuh"
#include "rank_row.cuh"

namespace {

constexpr int kChunk = 16;                  // splits per work item of the rank kernel
constexpr int kFits = kChunk * RS_NOPT;
constexpr int kKld = RS_MAXV + 1;           // padded row stride of K in shared memory
constexpr int kNReg = 10;                   // largest n solved by one thread in registers
constexpr int kNMid = 16;                   // largest n solved by one thread from shared memory
constexpr int kHist = RS_MAXPAIRS + 2;      // n = 0..32, plus one end slot
// Within the fits of one n, the bucket order is by the number of predictions c (0..64) the
// fit makes, inside each block's share of 4096 fits: a warp's 32 fits then mostly run
// prediction loops of one length.  Sort key n * kCntBins + c.
constexpr int kCntBins = RS_MAXV + 1;
constexpr int kKeys = (RS_MAXPAIRS + 1) * kCntBins;
constexpr int kBucketThreads = 512;
constexpr int kBucketPer = 8;                // fits per thread of the bucket kernel
static_assert(3 * 32 >= kCntBins, "a warp scans one n's counts three per lane");
static_assert(kBucketThreads / 32 * 2 >= RS_MAXPAIRS, "the bucket kernel's warps take two n each");
__host__ __device__ constexpr int tri(int n) { return n * (n + 1) / 2; }

// The a-th set bit (0-based) of x; x must have more than a set bits.
__device__ __forceinline__ int select_bit(uint64_t x, int a) {
    for (int i = 0; i < a; ++i) x &= x - 1;
    return __ffsll((long long)x) - 1;
}

// Gathering the bits of a 64-bit word at the positions of a fixed set into its low bits, in
// ascending order (a compress), in six rounds of shifts: round i moves each bit that still has
// to travel an odd multiple of 2^i places by 2^i.  compress_moves stores the set and its six
// move masks (the positions moved in each round, derived from the running count of the set's
// zeros below each bit -- the parallel-suffix construction of Hacker's Delight, Sec. 7-4);
// compress applies them.  A pair's training bit is T[b] & T[a] for its before and after
// slots; when both kinds of slot ascend with the pair index, compress(T, before set) &
// compress(T, after set) gives every pair's bit at once.
constexpr int kSetWords = 14;                // per (program, optimization): 2 x (set + 6 moves)

__device__ __forceinline__ void compress_moves(uint64_t m, uint64_t* out) {
    out[0] = m;
    uint64_t mk = ~m << 1;                   // bit k: a zero of the set lies below k
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        uint64_t mp = mk ^ (mk << 1);        // parity of the zeros below each bit
        mp ^= mp << 2;
        mp ^= mp << 4;
        mp ^= mp << 8;
        mp ^= mp << 16;
        mp ^= mp << 32;
        const uint64_t mv = mp & m;          // set bits that move in this round
        out[1 + i] = mv;
        m = (m ^ mv) | (mv >> (1 << i));
        mk &= ~mp;
    }
}

__device__ __forceinline__ uint64_t compress(uint64_t x, const uint64_t* c) {
    x &= c[0];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const uint64_t t = x & c[1 + i];
        x = (x ^ t) | (t >> (1 << i));
    }
    return x;
}

// ====================================================================== pair tables
// One block per program: the before/after pairs of each optimization in ascending order of
// the before slot, and their labels.  Tables: [P][6][32] (u8, u8, double), counts [P][6].
// Also, per program: cand[p][j] = slots whose mask lacks j (uint64), and for every slot t a
// summary of the actual log speedups of adding each j (Sec. 5: the measured speedup of the
// pair, used only for scoring).  Needs no Gram block: it may run beside the Gram.
__global__ void __launch_bounds__(64)
pairs_kernel(int P, const int64_t* __restrict__ row_off, const uint8_t* __restrict__ masks,
             const double* __restrict__ log_time, uint8_t* pb, uint8_t* pa, double* ylab,
             int* npair, uint64_t* cand, uint32_t* rowinfo, uint64_t* pset, uint8_t* psorted,
             int* dstatus) {
    __shared__ int8_t slot_of[RS_MAXV];
    __shared__ uint8_t msk[RS_MAXV];
    __shared__ double lt[RS_MAXV];
    const int p = blockIdx.x, tid = threadIdx.x;
    const int64_t r0 = row_off[p];
    const int V = (int)(row_off[p + 1] - r0);
    if (V < 1 || V > RS_MAXV) {
        if (tid < RS_NOPT) {
            npair[p * RS_NOPT + tid] = 0;
            cand[p * RS_NOPT + tid] = 0;
        }
        if (tid == 0) {
            psorted[p] = 0;
            rs_dev_flag(dstatus, RS_EDATA, p);
        }
        return;
    }
    slot_of[tid] = -1;
    if (tid < V) {
        msk[tid] = masks[r0 + tid] & 63;
        lt[tid] = log_time[r0 + tid];
    }
    __syncthreads();
    if (tid < V) slot_of[msk[tid]] = (int8_t)tid;
    // masks strictly ascending over the slots: then the after slots of a j's pairs ascend with
    // their before slots, and plan_fits may gather a split's pair bits set by set
    const int sorted = __syncthreads_and(tid == 0 || tid >= V || msk[tid] > msk[tid - 1]);
    if (tid == 0) psorted[p] = (uint8_t)sorted;
    // warp w takes optimizations w, w + 2, w + 4; its lanes take 32 slots at a time, and a
    // ballot places each pair after those of the lower slots
    const int warp = tid >> 5, lane = tid & 31;
    for (int j = warp; j < RS_NOPT; j += 2) {
        const int64_t base = ((int64_t)p * RS_NOPT + j) * RS_MAXPAIRS;
        int np = 0;
        uint64_t cm = 0, bset = 0, aset = 0;
        for (int v0 = 0; v0 < V; v0 += 32) {
            const int v = v0 + lane;
            const int m = v < V ? msk[v] : (1 << j);
            const bool c = !((m >> j) & 1);                  // slot v lacks j
            const int w = c ? slot_of[m | (1 << j)] : -1;
            const unsigned cb = __ballot_sync(0xffffffffu, c), pm = __ballot_sync(0xffffffffu, w >= 0);
            cm |= (uint64_t)cb << v0;
            const int at = np + __popc(pm & ((1u << lane) - 1u));
            if (w >= 0) {
                if (at < RS_MAXPAIRS) {
                    pb[base + at] = (uint8_t)v;
                    pa[base + at] = (uint8_t)w;
                    ylab[base + at] = lt[v] - lt[w];
                } else {
                    rs_dev_flag(dstatus, RS_EDATA, p);       // only possible with repeated masks
                }
            }
            np += __popc(pm);
            bset |= (uint64_t)pm << v0;
            const unsigned alo = __reduce_or_sync(0xffffffffu, w >= 0 && w < 32 ? 1u << w : 0u);
            const unsigned ahi = __reduce_or_sync(0xffffffffu, w >= 32 ? 1u << (w - 32) : 0u);
            aset |= (uint64_t)ahi << 32 | alo;
        }
        if (lane == 0) {
            npair[p * RS_NOPT + j] = np < RS_MAXPAIRS ? np : RS_MAXPAIRS;
            cand[p * RS_NOPT + j] = cm;
            uint64_t* ps = pset + ((int64_t)p * RS_NOPT + j) * kSetWords;
            compress_moves(bset, ps);
            compress_moves(aset, ps + kSetWords / 2);
        }
    }
    rowinfo[(int64_t)p * RS_MAXV + tid] = row_summary(tid, V, msk, lt, slot_of);
}

// dlam[p][t] = K_p[t][t] + lambda, the diagonal the solvers factor (one block per program).
__global__ void __launch_bounds__(64)
dlam_kernel(const int64_t* __restrict__ row_off, const double* __restrict__ K, double lambda, double* dlam) {
    const int p = blockIdx.x, t = threadIdx.x;
    const int V = (int)(row_off[p + 1] - row_off[p]);
    if (V >= 1 && V <= RS_MAXV && t < V)
        dlam[(int64_t)p * RS_MAXV + t] = K[(int64_t)p * RS_GRAM_LD * RS_GRAM_LD + t * RS_GRAM_LD + t] + lambda;
}

// ====================================================================== plan
constexpr int kPlanProgs = 8;                // programs whose pair tables a plan block stages
// One thread per split: the six pair masks of its fits (the pair loops run over one
// program's pair tables, uniform across a warp whose splits share the program), their sort
// keys n * kCntBins + c (c = the predictions the fit makes when predictions are wanted, else
// 0), the histogram of fit sizes (warp-aggregated), and the split's row records in slot order:
// the row's scoring summary | version mask << 30 | mask of the split's empty fits << 36.
__global__ void __launch_bounds__(256)
plan_fits_kernel(int P, const int64_t* __restrict__ row_off, const int64_t* __restrict__ split_off,
                 const uint64_t* __restrict__ tm, int64_t S, const uint8_t* __restrict__ pb,
                 const uint8_t* __restrict__ pa, const int* __restrict__ npair, uint32_t* fit_pm,
                 uint16_t* fit_key, unsigned* hist, int nmax, int* split_prog,
                 const int64_t* __restrict__ rec_offsets, int64_t rows_cap,
                 unsigned long long* row_info, const uint8_t* __restrict__ masks,
                 const uint32_t* __restrict__ rowinfo, const uint64_t* __restrict__ cand, int cand_all,
                 int count_preds, const uint64_t* __restrict__ pset, const uint8_t* __restrict__ psorted,
                 int* dstatus) {
    __shared__ unsigned h[kHist];
    // the tables of the block's first kPlanProgs programs (its splits' programs are
    // consecutive): pair slots [program][before / after][optimization][32], pair counts,
    // candidate masks, scoring summaries and version masks of the program's slots
    __shared__ __align__(16) uint8_t tab[kPlanProgs][2][RS_NOPT][RS_MAXPAIRS];
    __shared__ int snp[kPlanProgs][RS_NOPT];
    __shared__ uint64_t scand[kPlanProgs][RS_NOPT];
    __shared__ uint32_t sri[kPlanProgs][RS_MAXV];
    __shared__ uint8_t smk[kPlanProgs][RS_MAXV];
    __shared__ uint64_t sset[kPlanProgs][RS_NOPT][kSetWords];
    __shared__ uint8_t ssorted[kPlanProgs];
    __shared__ int p_first;
    if (threadIdx.x < kHist) h[threadIdx.x] = 0;
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int p = s < S ? rs_find_segment(split_off, P, s) : 0;
    if (threadIdx.x == 0) p_first = p;
    __syncthreads();
    {
        const int p0 = p_first, np_tab = P - p0 < kPlanProgs ? P - p0 : kPlanProgs;
        const int words = np_tab * RS_NOPT * RS_MAXPAIRS / 16;       // 16-byte words per table
        for (int w = threadIdx.x; w < 2 * words; w += blockDim.x) {
            const int t = w / words, r = w - t * words;               // table (before / after), word
            const int q = r / (RS_NOPT * RS_MAXPAIRS / 16), k = r - q * (RS_NOPT * RS_MAXPAIRS / 16);
            const uint8_t* src = (t ? pa : pb) + (int64_t)(p0 + q) * RS_NOPT * RS_MAXPAIRS;
            reinterpret_cast<uint4*>(&tab[q][t][0][0])[k] = __ldg(reinterpret_cast<const uint4*>(src) + k);
        }
        for (int i = threadIdx.x; i < np_tab * RS_MAXV; i += blockDim.x) {
            const int q = i / RS_MAXV, t = i - q * RS_MAXV, pq = p0 + q;
            const int64_t r0 = row_off[pq];
            sri[q][t] = rowinfo[(int64_t)pq * RS_MAXV + t];
            smk[q][t] = t < row_off[pq + 1] - r0 ? masks[r0 + t] : 0;
            if (t < RS_NOPT) {
                snp[q][t] = npair[pq * RS_NOPT + t];
                scand[q][t] = cand ? cand[pq * RS_NOPT + t] : 0ull;
            }
            if (t == 0) ssorted[q] = psorted[pq];
        }
        for (int i = threadIdx.x; i < np_tab * RS_NOPT * kSetWords; i += blockDim.x)
            (&sset[0][0][0])[i] = pset[(int64_t)p0 * RS_NOPT * kSetWords + i];
    }
    __syncthreads();
    if (s < S) {
        const int V = (int)(row_off[p + 1] - row_off[p]);
        const bool okV = V >= 1 && V <= RS_MAXV;
        split_prog[s] = p;
        const uint64_t full = okV ? rs_full_mask(V) : 0ull;
        const uint64_t T = tm[s] & full;
        int emptym = 0;
        // the program's pair tables: from shared memory, else (a block spanning more than
        // kPlanProgs programs) from global memory, as 16-byte vectors
        const int q = p - p_first;
        const bool st = q < kPlanProgs;
        const uint8_t* tb = st ? &tab[q][0][0][0] : pb + (int64_t)p * RS_NOPT * RS_MAXPAIRS;
        const uint8_t* ta = st ? &tab[q][1][0][0] : pa + (int64_t)p * RS_NOPT * RS_MAXPAIRS;
        const int* npp = st ? snp[q] : npair + p * RS_NOPT;
        const uint64_t* cp = st ? scand[q] : cand + p * RS_NOPT;
        const uint32_t* rip = st ? sri[q] : rowinfo + (int64_t)p * RS_MAXV;
        const uint8_t* mkp = st ? smk[q] : masks + row_off[p];
        const uint64_t* psp = st ? sset[q][0] : pset + (int64_t)p * RS_NOPT * kSetWords;
        const bool srt = okV && (st ? ssorted[q] : psorted[p]) != 0;
#pragma unroll 2
        for (int j = 0; j < RS_NOPT; ++j) {
            const int npj = okV ? npp[j] : 0;
            uint32_t pm = 0;
            if (srt) {
                // sorted masks: every pair's bit at once from the before and after slot sets
                const uint64_t* c = psp + j * kSetWords;
                pm = (uint32_t)(compress(T, c) & compress(T, c + kSetWords / 2));
            } else {
                const ulonglong2 vb[2] = {reinterpret_cast<const ulonglong2*>(tb + j * RS_MAXPAIRS)[0],
                                          reinterpret_cast<const ulonglong2*>(tb + j * RS_MAXPAIRS)[1]};
                const ulonglong2 va[2] = {reinterpret_cast<const ulonglong2*>(ta + j * RS_MAXPAIRS)[0],
                                          reinterpret_cast<const ulonglong2*>(ta + j * RS_MAXPAIRS)[1]};
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    if (8 * w >= npj) break;
                    const unsigned long long wb = (w & 1) ? vb[w >> 1].y : vb[w >> 1].x;
                    const unsigned long long wa = (w & 1) ? va[w >> 1].y : va[w >> 1].x;
                    uint32_t part = 0;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const unsigned sb = (unsigned)(wb >> (8 * e)) & 63u;
                        const unsigned sa = (unsigned)(wa >> (8 * e)) & 63u;
                        part |= (uint32_t)((T >> sb) & (T >> sa) & 1ull) << e;
                    }
                    const int keep = npj - 8 * w;             // pairs of this word that exist
                    if (keep < 8) part &= (1u << keep) - 1u;
                    pm |= part << (8 * w);
                }
            }
            int n = __popc(pm);
            if (n > nmax) {        // more pairs than the workspace was sized for
                rs_dev_flag(dstatus, RS_EDATA, -2);
                pm = 0;
                n = 0;
            }
            // c = the predictions the fit makes: its split's test rows that are candidates
            int c = 0;
            if (count_preds && n > 0) c = __popcll(~T & full & (cand_all ? full : cp[j]));
            const int key = n * kCntBins + c;
            fit_pm[s * RS_NOPT + j] = pm;
            fit_key[s * RS_NOPT + j] = (uint16_t)key;
            emptym |= (n == 0) << j;
            const unsigned grp = __match_any_sync(__activemask(), n);
            if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(&h[n], (unsigned)__popc(grp));
        }
        if (row_info && okV) {
            const uint64_t test = ~tm[s] & rs_full_mask(V);
            int64_t r = rec_offsets[s];
            for (uint64_t x = test; x && r < rows_cap; x &= x - 1, ++r) {
                const int t = __ffsll((long long)x) - 1;
                row_info[r] = (unsigned long long)rip[t] | ((unsigned long long)(mkp[t] & 63) << 30) |
                              ((unsigned long long)emptym << 36);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < kHist && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// Bucket starts from the histogram: positions of fits with n >= 1 ordered by n, and the
// offsets of their compact coefficient records (n + 1 doubles each).  Called by every
// thread of the block; warp 0 scans the 32 counts with shuffles.  Ends with a barrier.
__device__ __forceinline__ void bucket_tables(const unsigned* hist, long long* start, long long* cstart) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int n = lane + 1;
        const long long v = hist[n];
        const long long w = v * (n + 1);
        long long iv = v, iw = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long yv = __shfl_up_sync(0xffffffffu, iv, o);
            const long long yw = __shfl_up_sync(0xffffffffu, iw, o);
            if (lane >= o) {
                iv += yv;
                iw += yw;
            }
        }
        start[n] = iv - v;
        cstart[n] = iw - w;
        if (lane == 31) {
            start[RS_MAXPAIRS + 1] = iv;
            cstart[RS_MAXPAIRS + 1] = iw;
        }
        if (lane == 0) {
            start[0] = 0;
            cstart[0] = 0;
        }
    }
    __syncthreads();
}

// ====================================================================== solve, n <= kNReg
// Where the predictions of one fit go: the test rows of its split that are candidates for
// its optimization; row r of the split (r-th test slot in ascending order) is dst[r].
struct PredTarget {
    double* dst;          // prediction buffer row of this optimization + the split's first row
    uint64_t test;        // test slots of the split
    uint64_t cand;        // test slots to predict (candidates)
    int64_t room;         // rows left in the buffer from dst (guards a wrong size hint)
};

// One fit of n = N pairs in registers.  M = K_TT + lambda I = L D L^T (unit lower L, no
// square roots; reciprocal pivots by rcp_newton).  With t_y = L^-1 y and t_1 = L^-1 1:
//   1^T M^-1 y = t_1^T D^-1 t_y,  1^T M^-1 1 = t_1^T D^-1 t_1,  b = their ratio,
//   alpha = L^-T D^-1 (t_y - b t_1)   (one backward solve).
template <int N>
__device__ __forceinline__ int fit_fixed(const double* __restrict__ Kp, const uint8_t* __restrict__ pb,
                                         const double* __restrict__ yl, uint32_t pm,
                                         const double* __restrict__ dl, double* out, double (&ty)[N],
                                         double& b, int (&vb)[N]) {
    double t1[N], L[tri(N)], dinv[N];
    uint32_t x = pm;
#pragma unroll
    for (int a = 0; a < N; ++a) {
        const int q = __ffs(x) - 1;
        x &= x - 1;
        vb[a] = pb[q];
        ty[a] = yl[q];
    }
    if constexpr (N == 1) {
        // one pair: 1^T alpha = 0 forces alpha = 0, so b = y and every prediction is b
        if (!pos_finite(__ldg(dl + vb[0]))) return RS_FIT_NOTPD;
        b = ty[0];
        ty[0] = 0.0;
        if (out) {
            out[0] = b;
            out[1] = 0.0;
        }
        return finite_bits(b) ? RS_FIT_OK : RS_FIT_NONFINITE;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double c[N];                       // c_m = L_im d_m of the current row
#pragma unroll
        for (int k = 0; k < i; ++k) {
            double s = __ldg(Kp + vb[i] * RS_GRAM_LD + vb[k]);
#pragma unroll
            for (int m = 0; m < k; ++m) s = fma(-c[m], L[tri(k) + m], s);
            c[k] = s;
            L[tri(i) + k] = s * dinv[k];
        }
        double d = __ldg(dl + vb[i]);      // K[v][v] + lambda
#pragma unroll
        for (int m = 0; m < i; ++m) d = fma(-c[m], L[tri(i) + m], d);
        if (!pos_finite(d)) return RS_FIT_NOTPD;
        dinv[i] = rcp_newton(d);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {          // L t = rhs, unit diagonal, two right-hand sides
        t1[i] = 1.0;
#pragma unroll
        for (int k = 0; k < i; ++k) {
            ty[i] = fma(-L[tri(i) + k], ty[k], ty[i]);
            t1[i] = fma(-L[tri(i) + k], t1[k], t1[i]);
        }
    }
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const double sc = t1[i] * dinv[i];
        num = fma(sc, ty[i], num);
        den = fma(sc, t1[i], den);
    }
    b = num * rcp_newton(den);
#pragma unroll
    for (int i = 0; i < N; ++i) ty[i] = fma(-b, t1[i], ty[i]) * dinv[i];
#pragma unroll
    for (int i = N - 1; i >= 0; --i)       // L^T alpha = D^-1 (t_y - b t_1)
#pragma unroll
        for (int k = i + 1; k < N; ++k) ty[i] = fma(-L[tri(k) + i], ty[k], ty[i]);
    bool fin = finite_bits(b);
#pragma unroll
    for (int i = 0; i < N; ++i) fin = fin && finite_bits(ty[i]);
    if (out) {
        out[0] = b;
#pragma unroll
        for (int i = 0; i < N; ++i) out[1 + i] = ty[i];
    }
    return fin ? RS_FIT_OK : RS_FIT_NONFINITE;
}

// One fit of n = N pairs in registers (fit_fixed), then its predictions b + sum_a alpha_a
// K[t][v_a] for the candidate test rows of its split.
template <int N>
__device__ __forceinline__ int solve_fixed(const double* __restrict__ Kp, const uint8_t* __restrict__ pb,
                                           const double* __restrict__ yl, uint32_t pm,
                                           const double* __restrict__ dl, double* out,
                                           const PredTarget* pt) {
    double al[N], b = 0.0;
    int vb[N];
    const int st = fit_fixed<N>(Kp, pb, yl, pm, dl, out, al, b, vb);
    if (st != RS_FIT_OK || !pt) return st;
    uint64_t cm = pt->cand;
    if constexpr (N == 1) {                // with one pair alpha = 0: every prediction is b
        for (; cm; cm &= cm - 1) {
            const int t = __ffsll((long long)cm) - 1;
            const int r = __popcll(pt->test & ((1ull << t) - 1ull));
            if (r < pt->room) pt->dst[r] = b;
        }
    } else if (cm) {
        // software pipeline: the Gram entries of the next candidate row are loaded while the
        // current row's dot product runs
        int t = __ffsll((long long)cm) - 1;
        double kv[N];
#pragma unroll
        for (int a = 0; a < N; ++a) kv[a] = __ldg(Kp + t * RS_GRAM_LD + vb[a]);
        for (;;) {
            cm &= cm - 1;
            const int tn = cm ? __ffsll((long long)cm) - 1 : t;
            double kn[N];
#pragma unroll
            for (int a = 0; a < N; ++a) kn[a] = __ldg(Kp + tn * RS_GRAM_LD + vb[a]);
            double yh = b;
#pragma unroll
            for (int a = 0; a < N; ++a) yh = fma(al[a], kv[a], yh);
            const int r = __popcll(pt->test & ((1ull << t) - 1ull));
            if (r < pt->room) pt->dst[r] = yh;
            if (!cm) break;
            t = tn;
#pragma unroll
            for (int a = 0; a < N; ++a) kv[a] = kn[a];
        }
    }
    return st;
}

template <int N, int NHI>
__device__ __forceinline__ int solve_dispatch(int n, const double* Kp, const uint8_t* pb, const double* yl,
                                              uint32_t pm, const double* dl, double* out,
                                              const PredTarget* pt) {
    if constexpr (N >= NHI) {
        return solve_fixed<N>(Kp, pb, yl, pm, dl, out, pt);
    } else {
        if (n == N) return solve_fixed<N>(Kp, pb, yl, pm, dl, out, pt);
        return solve_dispatch<N + 1, NHI>(n, Kp, pb, yl, pm, dl, out, pt);
    }
}

struct SolveArgs {
    int P;
    const int64_t* split_off;
    const int* split_prog;
    const double* K;
    const uint8_t* pb;
    const double* ylab;
    const uint32_t* fit_pm;
    const uint16_t* fit_key;
    const uint4* recs;    // [S*6] in bucket order: fit index, program, pair mask, versions
    const unsigned* hist;
    const int64_t* fit_off;
    double* coef;         // compact records, or the caller's [S][6][33] array
    int coef_user;
    uint8_t* status;
    double lambda;
    const double* dlam;   // [P][64] K[t][t] + lambda
    unsigned long long* counters;
    // predictions (batched predict/rank only; predbuf == nullptr for fits alone)
    const int64_t* row_off;
    const uint64_t* train_masks;
    const int64_t* rec_offsets;
    const uint64_t* cand;
    double* predbuf;      // [6][PS]: plane j holds the predictions of optimization j
    int64_t R;            // rows of the buffer (the bound every write is checked against)
    int64_t PS;           // plane stride (rows), even
    int flags;
    int* dstatus;
    // refinement through Z (RS_REFINE_X)
    const double* Z;
    const int64_t* x_offsets;
    const int32_t* feat_width;
    int max_feat;
    int order;            // 0: largest fits first; 1: alternate ranges from both ends
    unsigned long long* row_info;   // [R] the rank pass's row records (with predictions)
};

__device__ __forceinline__ bool pred_target_v(const SolveArgs& a, int64_t s, int j, int p, int V, PredTarget& pt) {
    if (!a.predbuf) return false;
    const uint64_t full = rs_full_mask(V);
    pt.test = ~a.train_masks[s] & full;
    pt.cand = pt.test & ((a.flags & RS_RANK_ALL) ? full : a.cand[p * RS_NOPT + j]);
    const int64_t r0 = a.rec_offsets[s];
    pt.dst = a.predbuf + (int64_t)j * a.PS + r0;
    pt.room = a.R - r0;
    if (r0 + __popcll(pt.test) > a.R) rs_dev_flag(a.dstatus, RS_EDATA, -3);
    return true;
}
__device__ __forceinline__ bool pred_target(const SolveArgs& a, int64_t s, int j, int p, PredTarget& pt) {
    return pred_target_v(a, s, j, p, (int)(a.row_off[p + 1] - a.row_off[p]), pt);
}

// A fit (s, j) that failed sets bit 36 + j in the row records of its candidate rows, beside the
// fits without a training pair: the rank pass leaves optimization j out of those rows and reads
// no fit status.
__device__ __forceinline__ void mark_failed(const SolveArgs& a, int64_t s, int j, const PredTarget& pt) {
    unsigned long long* info = a.row_info + a.rec_offsets[s];
    for (uint64_t cm = pt.cand; cm; cm &= cm - 1) {
        const int t = __ffsll((long long)cm) - 1;
        const int r = __popcll(pt.test & ((1ull << t) - 1ull));
        if (r < pt.room) atomicOr(info + r, 1ull << (36 + j));
    }
}

__device__ __forceinline__ void finish_record(const SolveArgs& a, int64_t f, int n, int st, double* out) {
    if (out && st != RS_FIT_OK) {
        out[0] = nan_d();
        for (int e = 1; e <= n; ++e) out[e] = 0.0;
    }
    if (out && a.coef_user)
        for (int e = n + 1; e < RS_COEF_STRIDE; ++e) out[e] = 0.0;
    a.status[f] = (uint8_t)st;
}

// Where a fit's coefficients go: the caller's [S][6][33] array, else (fits without
// predictions) the compact records; the predict-and-rank path keeps none.
__device__ __forceinline__ double* coef_out(const SolveArgs& a, int64_t f) {
    if (a.coef_user) return a.coef + f * RS_COEF_STRIDE;
    return a.predbuf ? nullptr : a.coef + a.fit_off[f];
}

// ====================================================================== bucket
// Counting sort of the fits by n, and by c inside each block's share: a block of 4096 fits
// counts them per (n, c) in shared memory, reserves one range per n with a single global
// atomic, and places its fits' records inside it in ascending c (fit index, program, pair
// mask, version count: what a solver needs first).  The order inside a bucket is immaterial
// to the results: every result goes to its fit's own place.
// A fit without a training pair (n = 0) is finished here (status RS_FIT_EMPTY); the rank
// pass knows it from the row records.
__global__ void __launch_bounds__(kBucketThreads, 2)
bucket_fits_kernel(int64_t S6, const uint16_t* __restrict__ fit_key, const unsigned* __restrict__ hist,
                   unsigned* cursor, uint4* recs, int64_t* fit_off, uint8_t* status, double* coef_user,
                   unsigned long long* counters, const uint32_t* __restrict__ fit_pm,
                   const int* __restrict__ split_prog, const int64_t* __restrict__ row_off) {
    __shared__ long long start[kHist], cstart[kHist];
    __shared__ unsigned lcount[kKeys];       // fits per (n, c); then their offsets inside n's range
    __shared__ unsigned lbase[kHist];
    for (int i = threadIdx.x; i < kKeys; i += kBucketThreads) lcount[i] = 0;
    bucket_tables(hist, start, cstart);      // (ends with a barrier)
    const int64_t f0 = (int64_t)blockIdx.x * (kBucketThreads * kBucketPer) + threadIdx.x;
    int key[kBucketPer];
    unsigned local[kBucketPer];
    uint4 rec[kBucketPer];                   // each fit's record, loaded before the block's scan
#pragma unroll
    for (int q = 0; q < kBucketPer; ++q) {
        const int64_t f = f0 + (int64_t)q * kBucketThreads;
        key[q] = f < S6 ? fit_key[f] : 0;
        local[q] = key[q] >= kCntBins ? atomicAdd(&lcount[key[q]], 1u) : 0u;
        rec[q] = make_uint4((unsigned)f, 0u, 0u, 0u);
        if (key[q] >= kCntBins) {
            const int p = split_prog[f / RS_NOPT];
            rec[q].y = (unsigned)p;
            rec[q].z = fit_pm[f];
            rec[q].w = (unsigned)(row_off[p + 1] - row_off[p]);
        }
    }
    __syncthreads();
    // warp w scans the counts of n = w + 1 and n = w + 17: exclusive offsets over c, and the
    // block's range of that n
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int n = warp + 1; n <= RS_MAXPAIRS; n += kBucketThreads / 32) {
        unsigned* row = lcount + n * kCntBins;
        unsigned v[3], sum = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int c = 3 * lane + i;
            v[i] = c < kCntBins ? row[c] : 0u;
            sum += v[i];
        }
        unsigned incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        unsigned run = incl - sum;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int c = 3 * lane + i;
            if (c < kCntBins) {
                row[c] = run;
                run += v[i];
            }
        }
        const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
        if (lane == 0) lbase[n] = total ? atomicAdd(&cursor[n], total) : 0u;
    }
    __syncthreads();
    unsigned empty = 0;
#pragma unroll
    for (int q = 0; q < kBucketPer; ++q) {
        const int64_t f = f0 + (int64_t)q * kBucketThreads;
        if (f >= S6) break;
        const int n = key[q] / kCntBins;
        if (n == 0) {
            if (fit_off) fit_off[f] = -1;
            status[f] = RS_FIT_EMPTY;
            ++empty;
            if (coef_user) {
                double* o = coef_user + f * RS_COEF_STRIDE;
                o[0] = nan_d();
                for (int e = 1; e < RS_COEF_STRIDE; ++e) o[e] = 0.0;
            }
        } else {
            const long long pos = start[n] + lbase[n] + lcount[key[q]] + local[q];
            recs[pos] = rec[q];              // the solver's whole first round trip in 16 bytes
            if (fit_off) fit_off[f] = cstart[n] + (pos - start[n]) * (n + 1);
        }
    }
    if (counters) {
        const unsigned e = __reduce_add_sync(0xffffffffu, empty);
        if (lane == 0 && e) atomicAdd(counters + 10, (unsigned long long)e);
    }
}

// Dynamic work distribution: a warp takes the next 32 positions of its range from a global
// counter; the following range is requested before the current one is solved, so the
// atomic's latency is hidden.  Kernels sharing the GPU with another one (or with a late
// block) thus never leave a statically assigned share behind.
__device__ __forceinline__ unsigned long long take32(unsigned long long* ctr) {
    unsigned long long got = 0;
    if ((threadIdx.x & 31) == 0) got = atomicAdd(ctr, 32ull);
    return got;
}

__device__ __forceinline__ void count_status(const SolveArgs& a, int st, bool active) {
    if (!a.counters) return;
    const unsigned lane = threadIdx.x & 31;
    const unsigned ok = __reduce_add_sync(0xffffffffu, active && st == RS_FIT_OK);
    const unsigned np = __reduce_add_sync(0xffffffffu, active && st == RS_FIT_NOTPD);
    const unsigned nf = __reduce_add_sync(0xffffffffu, active && st == RS_FIT_NONFINITE);
    if (lane == 0) {
        if (ok) atomicAdd(a.counters + 9, (unsigned long long)ok);
        if (np) atomicAdd(a.counters + 11, (unsigned long long)np);
        if (nf) atomicAdd(a.counters + 12, (unsigned long long)nf);
    }
}

// Fits with NLO <= n <= NHI, one per thread, in bucket order (n is warp-uniform except at
// bucket boundaries).  Warps take ranges of 32 bucket positions from a global counter.
// Order 0: from the top of the range down -- the largest fits first, the cheapest last, so
// the final ranges (the tail of the kernel) are short.  Order 1: the q-th range taken comes
// alternately from the top (largest fits, descending) and from the bottom (smallest fits,
// ascending), meeting in the middle: the FP64-light fits, whose time goes to memory
// latency, run beside FP64-heavy ones instead of in a phase of their own.
template <int NLO, int NHI, int MINB>
__global__ void __launch_bounds__(128, MINB)
solve_small_kernel(const SolveArgs a, unsigned long long* work) {
    __shared__ long long start[kHist], cstart[kHist];
    bucket_tables(a.hist, start, cstart);
    const long long lo = start[NLO], hi = start[NHI + 1];
    const int lane = threadIdx.x & 31;
    const long long nr = (hi - lo + 31) >> 5;           // ranges
    const long long split = hi - 32 * ((nr + 1) >> 1);  // top ranges cover [split, hi)
    const bool both = a.order == 1;
    auto position = [&](long long b) {
        const long long q = (b - lo) >> 5;
        if (!both) return hi - 1 - (b - lo) - lane;
        if ((q & 1) == 0) return hi - 1 - 32 * (q >> 1) - lane;
        const long long p = lo + 32 * (q >> 1) + lane;
        return p < split ? p : lo - 1;                   // past the top ranges: inactive
    };
    // two ranges ahead: the record of the next range is loaded while this one is solved
    long long base = lo + (long long)__shfl_sync(0xffffffffu, take32(work), 0);
    unsigned long long got = take32(work);
    uint4 rec = make_uint4(0, 0, 0, 0);
    if (base < hi && position(base) >= lo) rec = a.recs[position(base)];
    while (base < hi) {
        const long long next = lo + (long long)__shfl_sync(0xffffffffu, got, 0);
        got = take32(work);
        uint4 nrec = make_uint4(0, 0, 0, 0);
        if (next < hi && position(next) >= lo) nrec = a.recs[position(next)];
        const long long pos = position(base);
        const bool active = pos >= lo;
        int st = RS_FIT_OK;
        if (active) {
            int n = NLO;
            while (start[n + 1] <= pos) ++n;
            const int64_t f = rec.x;
            const int64_t s = f / RS_NOPT;
            const int j = (int)(f - s * RS_NOPT);
            const int p = (int)rec.y;
            const double* Kp = a.K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
            const int64_t pbase = ((int64_t)p * RS_NOPT + j) * RS_MAXPAIRS;
            double* out = coef_out(a, f);
            PredTarget ptv;
            const PredTarget* pt = pred_target_v(a, s, j, p, (int)rec.w, ptv) ? &ptv : nullptr;
            st = solve_dispatch<NLO, NHI>(n, Kp, a.pb + pbase, a.ylab + pbase, rec.z,
                                          a.dlam + (int64_t)p * RS_MAXV, out, pt);
            if (st != RS_FIT_OK && pt) mark_failed(a, s, j, *pt);
            finish_record(a, f, n, st, out);
        }
        count_status(a, st, active);
        base = next;
        rec = nrec;
    }
}

// ====================================================================== IBK (Sec. 3.4)

// Mean label of the kIbkK pairs of pm (more than kIbkK of them) whose before versions are
// nearest to a test row, Dt being that row of the distance block and pb the before slot of
// each pair.  The list is ordered by (distance, pair index): distances are non-negative, so
// their bit patterns order like the values, and a pair replaces the last entry only when
// strictly nearer.  The chosen labels are summed in ascending pair index.
__device__ __forceinline__ double ibk_nearest_mean(uint32_t pm, const double* __restrict__ Dt,
                                                   const uint8_t* pb, const double* yl) {
    unsigned long long kd[kIbkK];
    int kq[kIbkK];
#pragma unroll
    for (int i = 0; i < kIbkK; ++i) {
        kd[i] = ~0ull;
        kq[i] = 0;
    }
    for (uint32_t x = pm; x; x &= x - 1) {
        const int q = __ffs(x) - 1;
        ibk_insert(kd, kq, (unsigned long long)__double_as_longlong(__ldg(Dt + pb[q])), q);
    }
    uint32_t chosen = 0;
#pragma unroll
    for (int i = 0; i < kIbkK; ++i) chosen |= 1u << kq[i];
    double sum = 0.0;
    for (uint32_t x = chosen; x; x &= x - 1) sum += yl[__ffs(x) - 1];
    return sum / (double)kIbkK;
}

// The instance-based learner, one fit per thread (bucket order, dynamic work, largest n
// first).  K is the distance block D_p[t][v] = |z_t - z_v|^2.  For each candidate test row t
// the prediction is the mean label of the kIbkK training pairs nearest to t
// (ibk_nearest_mean).  With at most kIbkK pairs every pair is a neighbour, whatever t, so
// the mean is formed once.
__global__ void __launch_bounds__(128)
ibk_kernel(const SolveArgs a, int nmax, unsigned long long* work) {
    __shared__ long long start[kHist], cstart[kHist];
    bucket_tables(a.hist, start, cstart);
    const long long lo = start[1], hi = start[nmax + 1];
    unsigned long long got = take32(work);
    long long base = lo + (long long)__shfl_sync(0xffffffffu, got, 0);
    while (base < hi) {
        got = take32(work);
        const long long pos = hi - 1 - (base - lo) - (threadIdx.x & 31);
        const bool active = pos >= lo;
        if (active) {
            int n = 1;
            while (start[n + 1] <= pos) ++n;
            const uint4 rec = a.recs[pos];
            const int64_t f = rec.x;
            const int64_t s = f / RS_NOPT;
            const int j = (int)(f - s * RS_NOPT);
            const int p = (int)rec.y;
            const double* Dp = a.K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
            const int64_t pbase = ((int64_t)p * RS_NOPT + j) * RS_MAXPAIRS;
            const uint32_t pm = rec.z;
            const double* yl = a.ylab + pbase;
            PredTarget pt;
            if (pred_target(a, s, j, p, pt)) {
                if (n <= kIbkK) {
                    double sum = 0.0;
                    for (uint32_t x = pm; x; x &= x - 1) sum += yl[__ffs(x) - 1];
                    const double mean = sum / (double)n;
                    for (uint64_t cm = pt.cand; cm; cm &= cm - 1) {
                        const int t = __ffsll((long long)cm) - 1;
                        const int r = __popcll(pt.test & ((1ull << t) - 1ull));
                        if (r < pt.room) pt.dst[r] = mean;
                    }
                } else {
                    const uint8_t* pb = a.pb + pbase;
                    for (uint64_t cm = pt.cand; cm; cm &= cm - 1) {
                        const int t = __ffsll((long long)cm) - 1;
                        const double mean = ibk_nearest_mean(pm, Dp + t * RS_GRAM_LD, pb, yl);
                        const int r = __popcll(pt.test & ((1ull << t) - 1ull));
                        if (r < pt.room) pt.dst[r] = mean;
                    }
                }
            }
            finish_record(a, f, n, RS_FIT_OK, a.coef_user ? a.coef + f * RS_COEF_STRIDE : nullptr);
        }
        count_status(a, RS_FIT_OK, active);
        base = lo + (long long)__shfl_sync(0xffffffffu, got, 0);
    }
}

// One fit of kNReg < n <= nmax pairs per thread, the same arithmetic as solve_fixed with
// run-time loops.  The factor and the work vectors live in shared memory, element-major
// across the 32 lanes of the warp (element e of this lane at W[32 e]): every access of a
// warp touches 32 distinct banks.  Layout per lane: L (tri(nmax)), D^-1, t_y, t_1 (nmax each).
__device__ int solve_var(int n, int nmax, const double* __restrict__ Kp, const uint8_t* __restrict__ pb,
                         const double* __restrict__ yl, uint32_t pm, const double* __restrict__ dl,
                         double* out, const PredTarget* pt, double* W, int* VB) {
    const int oD = tri(nmax), oY = oD + nmax, oT = oY + nmax;
#define LW(e) W[(size_t)(e) * 32]
    uint32_t x = pm;
    for (int q = 0; q < n; ++q) {
        const int bit = __ffs(x) - 1;
        x &= x - 1;
        VB[q * 32] = pb[bit];
        LW(oY + q) = yl[bit];
    }
    for (int i = 0; i < n; ++i) {
        const double* Ki = Kp + VB[i * 32] * RS_GRAM_LD;
        for (int k = 0; k < i; ++k) {          // c_k of row i, kept in the slot of L(i, k)
            double s = __ldg(Ki + VB[k * 32]);
            for (int m = 0; m < k; ++m) s = fma(-LW(tri(i) + m), LW(tri(k) + m), s);
            LW(tri(i) + k) = s;
        }
        double d = __ldg(dl + VB[i * 32]);
        for (int m = 0; m < i; ++m) {          // L(i, m) = c_m / d_m; d_i = M_ii - sum c_m L(i, m)
            const double c = LW(tri(i) + m);
            const double l = c * LW(oD + m);
            LW(tri(i) + m) = l;
            d = fma(-c, l, d);
        }
        if (!pos_finite(d)) return RS_FIT_NOTPD;
        LW(oD + i) = rcp_newton(d);
    }
    for (int i = 0; i < n; ++i) {              // L t = rhs, two right-hand sides
        double ty = LW(oY + i), t1 = 1.0;
        for (int k = 0; k < i; ++k) {
            const double l = LW(tri(i) + k);
            ty = fma(-l, LW(oY + k), ty);
            t1 = fma(-l, LW(oT + k), t1);
        }
        LW(oY + i) = ty;
        LW(oT + i) = t1;
    }
    double num = 0.0, den = 0.0;
    for (int i = 0; i < n; ++i) {
        const double sc = LW(oT + i) * LW(oD + i);
        num = fma(sc, LW(oY + i), num);
        den = fma(sc, LW(oT + i), den);
    }
    const double b = num * rcp_newton(den);
    for (int i = 0; i < n; ++i) LW(oY + i) = fma(-b, LW(oT + i), LW(oY + i)) * LW(oD + i);
    for (int i = n - 1; i >= 0; --i) {         // L^T alpha = D^-1 (t_y - b t_1)
        double v = LW(oY + i);
        for (int k = i + 1; k < n; ++k) v = fma(-LW(tri(k) + i), LW(oY + k), v);
        LW(oY + i) = v;
    }
    bool fin = finite_bits(b);
    for (int i = 0; i < n; ++i) fin = fin && finite_bits(LW(oY + i));
    if (out) {
        out[0] = b;
        for (int i = 0; i < n; ++i) out[1 + i] = LW(oY + i);
    }
    if (!fin) return RS_FIT_NONFINITE;
    if (pt)
        for (uint64_t cm = pt->cand; cm; cm &= cm - 1) {
            const int t = __ffsll((long long)cm) - 1;
            const int r = __popcll(pt->test & ((1ull << t) - 1ull));
            const double* Kt = Kp + t * RS_GRAM_LD;
            double yh = b;
            for (int q = 0; q < n; ++q) yh = fma(LW(oY + q), __ldg(Kt + VB[q * 32]), yh);
            if (r < pt->room) pt->dst[r] = yh;
        }
#undef LW
    return RS_FIT_OK;
}

// Shared memory of solve_mid_kernel per warp, in bytes.
__host__ __device__ constexpr size_t mid_warp_bytes(int nmax) {
    return (size_t)32 * ((size_t)(tri(nmax) + 3 * nmax) * sizeof(double) + (size_t)nmax * sizeof(int));
}

// Fits with kNReg < n, one per thread (solve_var), dynamic work distribution.
__global__ void __launch_bounds__(128)
solve_mid_kernel(const SolveArgs a, int nmax, unsigned long long* work) {
    extern __shared__ __align__(16) double dsm[];
    __shared__ long long start[kHist], cstart[kHist];
    bucket_tables(a.hist, start, cstart);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = tri(nmax) + 3 * nmax;
    double* W = dsm + (size_t)warp * per * 32 + lane;
    int* VB = reinterpret_cast<int*>(dsm + (size_t)(blockDim.x >> 5) * per * 32) + (size_t)warp * nmax * 32 + lane;
    const long long lo = start[kNReg + 1], hi = start[nmax + 1];
    unsigned long long got = take32(work);
    long long base = lo + (long long)__shfl_sync(0xffffffffu, got, 0);
    while (base < hi) {
        got = take32(work);
        const long long pos = hi - 1 - (base - lo) - lane;
        const bool active = pos >= lo;
        int st = RS_FIT_OK;
        if (active) {
            int n = kNReg + 1;
            while (start[n + 1] <= pos) ++n;
            const uint4 rec = a.recs[pos];
            const int64_t f = rec.x;
            const int64_t s = f / RS_NOPT;
            const int j = (int)(f - s * RS_NOPT);
            const int p = (int)rec.y;
            const double* Kp = a.K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
            const int64_t pbase = ((int64_t)p * RS_NOPT + j) * RS_MAXPAIRS;
            double* out = coef_out(a, f);
            PredTarget ptv;
            const PredTarget* pt = pred_target(a, s, j, p, ptv) ? &ptv : nullptr;
            st = solve_var(n, nmax, Kp, a.pb + pbase, a.ylab + pbase, rec.z,
                           a.dlam + (int64_t)p * RS_MAXV, out, pt, W, VB);
            if (st != RS_FIT_OK && pt) mark_failed(a, s, j, *pt);
            finish_record(a, f, n, st, out);
        }
        count_status(a, st, active);
        base = lo + (long long)__shfl_sync(0xffffffffu, got, 0);
    }
}

// ====================================================================== solve, one fit per warp
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// One step of iterative refinement through the feature vectors, for a Gram block that is
// only approximately Z Z^T (the tensor-core form): the exact bordered residual
//   r_a = y_a - b - lambda alpha_a - z_{v_a} . beta,  r_0 = -sum_a alpha_a,  beta = sum_a alpha_a z_{v_a}
// is computed in FP64 from Z, the correction solves the same factored system, and the
// predictions are b + z_t . beta (through Z, not through the Gram block).
struct RefineCtx {
    const double* Zp;     // the program's standardized rows, [V][F]
    int F;
    double* beta;         // per-warp shared buffer of F doubles
    double* sh;           // per-warp shared buffer of 64 doubles (coefficients)
    int* vsh;             // per-warp shared buffer of 32 ints (pair slots)
};

// Lane a owns row a (a < n <= 32).  K is read with leading dimension ld.  Lsh: [32][33].
// Writes b to coef[0] and alpha to coef[1..n]; returns a warp-uniform status.
__device__ int fit_warp(int n, uint32_t pm, const uint8_t* pair_b, const double* ylab,
                        const double* K, int ld, double lambda, double* Lsh, double* coef,
                        const PredTarget* pt = nullptr, const RefineCtx* rf = nullptr) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < n;
    int v = 0;
    double y = 0.0;
    if (act) {
        const int q = select_bit(pm, lane);
        v = pair_b[q];
        y = ylab[q];
    }
    // stage row a of M = K_TT + lambda I (lower triangle) in Lsh: independent loads
    for (int b = 0; b < n; ++b) {
        const int vb = __shfl_sync(0xffffffffu, v, b);
        if (act && b <= lane) Lsh[lane * 33 + b] = K[v * ld + vb] + (b == lane ? lambda : 0.0);
    }
    __syncwarp();
    double rinv = 0.0;
    for (int jj = 0; jj < n; ++jj) {           // left-looking, in place
        double s = 0.0;
        if (act && lane >= jj) {
            s = Lsh[lane * 33 + jj];
            for (int m = 0; m < jj; ++m) s = fma(-Lsh[lane * 33 + m], Lsh[jj * 33 + m], s);
        }
        const double d = __shfl_sync(0xffffffffu, s, jj);
        if (!pos_finite(d)) return RS_FIT_NOTPD;
        const double r = rsqrt_newton(d);
        if (lane == jj) rinv = r;
        else if (act && lane > jj) Lsh[lane * 33 + jj] = s * r;
        __syncwarp();
    }
    double u = y, w = act ? 1.0 : 0.0;
    for (int kk = 0; kk < n; ++kk) {          // forward: L t = rhs
        const double r = __shfl_sync(0xffffffffu, rinv, kk);
        const double uk = __shfl_sync(0xffffffffu, u, kk) * r;
        const double wk = __shfl_sync(0xffffffffu, w, kk) * r;
        if (lane == kk) {
            u = uk;
            w = wk;
        } else if (act && lane > kk) {
            const double l = Lsh[lane * 33 + kk];
            u = fma(-l, uk, u);
            w = fma(-l, wk, w);
        }
    }
    for (int kk = n - 1; kk >= 0; --kk) {     // backward: L^T x = t
        const double r = __shfl_sync(0xffffffffu, rinv, kk);
        const double uk = __shfl_sync(0xffffffffu, u, kk) * r;
        const double wk = __shfl_sync(0xffffffffu, w, kk) * r;
        if (lane == kk) {
            u = uk;
            w = wk;
        } else if (lane < kk) {
            const double l = Lsh[kk * 33 + lane];
            u = fma(-l, uk, u);
            w = fma(-l, wk, w);
        }
    }
    double su = act ? u : 0.0, sw = act ? w : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
    }
    double b = su / sw;
    double al = fma(-b, w, u);
    int fin = __all_sync(0xffffffffu, !act || finite_bits(al)) && finite_bits(b);
    if (rf && fin) {
        const int F = rf->F;
        const double* Zp = rf->Zp;
        double* beta = rf->beta;
        if (act) {
            rf->sh[lane] = al;
            rf->vsh[lane] = v;
        }
        __syncwarp();
        for (int f = lane; f < F; f += 32) {          // beta = sum_a alpha_a z_{v_a}
            double acc = 0.0;
            for (int q = 0; q < n; ++q) acc = fma(rf->sh[q], Zp[(int64_t)rf->vsh[q] * F + f], acc);
            beta[f] = acc;
        }
        __syncwarp();
        double ra = 0.0;                              // z_{v_q} . beta, lane q keeps its own
        for (int q = 0; q < n; ++q) {
            double part = 0.0;
            for (int f = lane; f < F; f += 32) part = fma(Zp[(int64_t)rf->vsh[q] * F + f], beta[f], part);
            part = warp_sum(part);
            if (lane == q) ra = part;
        }
        ra = act ? y - b - lambda * al - ra : 0.0;
        const double r0 = -warp_sum(act ? al : 0.0);
        double uu = ra;
        for (int kk = 0; kk < n; ++kk) {              // forward with the same factor
            const double r = __shfl_sync(0xffffffffu, rinv, kk);
            const double uk = __shfl_sync(0xffffffffu, uu, kk) * r;
            if (lane == kk) uu = uk;
            else if (act && lane > kk) uu = fma(-Lsh[lane * 33 + kk], uk, uu);
        }
        for (int kk = n - 1; kk >= 0; --kk) {         // backward
            const double r = __shfl_sync(0xffffffffu, rinv, kk);
            const double uk = __shfl_sync(0xffffffffu, uu, kk) * r;
            if (lane == kk) uu = uk;
            else if (lane < kk) uu = fma(-Lsh[kk * 33 + lane], uk, uu);
        }
        const double db = (warp_sum(act ? uu : 0.0) - r0) / warp_sum(act ? w : 0.0);
        const double da = act ? fma(-db, w, uu) : 0.0;
        al += da;
        b += db;
        if (act) rf->sh[32 + lane] = da;
        __syncwarp();
        for (int f = lane; f < F; f += 32) {          // beta += sum_a dalpha_a z_{v_a}
            double acc = beta[f];
            for (int q = 0; q < n; ++q) acc = fma(rf->sh[32 + q], Zp[(int64_t)rf->vsh[q] * F + f], acc);
            beta[f] = acc;
        }
        __syncwarp();
        fin = __all_sync(0xffffffffu, !act || finite_bits(al)) && finite_bits(b);
    }
    if (coef) {
        if (act) coef[1 + lane] = al;
        if (lane == 0) coef[0] = b;
    }
    __syncwarp();
    if (!fin) return RS_FIT_NONFINITE;
    if (pt && rf) {                           // predictions through Z: b + z_t . beta
        for (uint64_t cm = pt->cand; cm; cm &= cm - 1) {
            const int t = __ffsll((long long)cm) - 1;
            double part = 0.0;
            for (int f = lane; f < rf->F; f += 32) part = fma(rf->Zp[(int64_t)t * rf->F + f], rf->beta[f], part);
            part = warp_sum(part);
            if (lane == 0) {
                const int r = __popcll(pt->test & ((1ull << t) - 1ull));
                if (r < pt->room) pt->dst[r] = b + part;
            }
        }
        __syncwarp();
    } else if (pt) {                          // predictions, one candidate row per lane
        const int nc = __popcll(pt->cand);
        for (int r0 = 0; r0 < nc; r0 += 32) {
            const bool mine = r0 + lane < nc;
            int t = 0;
            if (mine) t = select_bit(pt->cand, r0 + lane);
            double yh = b;
            for (int q = 0; q < n; ++q) {
                const double aq = __shfl_sync(0xffffffffu, al, q);
                const int vq = __shfl_sync(0xffffffffu, v, q);
                if (mine) yh = fma(aq, K[t * ld + vq], yh);
            }
            if (mine) {
                const int r = __popcll(pt->test & ((1ull << t) - 1ull));
                if (r < pt->room) pt->dst[r] = yh;
            }
        }
    }
    return RS_FIT_OK;
}

// One fit per warp for the batched form without refinement: lane a owns row a (a < n <= 32)
// of M = K_TT + lambda I = L D L^T (unit lower L, no square roots), factored left-looking in
// shared memory.  Lsh holds L ([32][33]); Ush holds U = L D by rows, the operand every lane
// reads when a column is formed: s_i = M_i,j - sum_m L_i,m U_j,m, d_j = s_j, L_i,j = s_i / d_j,
// U_i,j = s_i.  Then t_y = L^-1 y, t_1 = L^-1 1 (one FMA per lane per step each), b = t_1^T D^-1
// t_y / t_1^T D^-1 t_1 and alpha = L^-T D^-1 (t_y - b t_1), the solve_fixed arithmetic with
// lanes for rows.  Predictions: one candidate row per lane.  Returns a warp-uniform status.
__device__ int fit_warp_ldl(int n, uint32_t pm, const uint8_t* pair_b, const double* ylab, const double* K,
                            const double* dl, double* Lsh, double* Ush, double* coef, const PredTarget* pt) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < n;
    int v = 0;
    double y = 0.0;
    if (act) {
        const int q = select_bit(pm, lane);
        v = pair_b[q];
        y = ylab[q];
    }
    for (int b = 0; b < n; ++b) {            // row a of M below the diagonal: independent loads
        const int vb = __shfl_sync(0xffffffffu, v, b);
        if (act && b < lane) Lsh[lane * 33 + b] = __ldg(K + v * RS_GRAM_LD + vb);
    }
    double dinv = 0.0;                       // lane a: 1 / d_a
    __syncwarp();
    for (int jj = 0; jj < n; ++jj) {
        double sv = 0.0;
        if (act && lane >= jj) {
            sv = lane == jj ? __ldg(dl + v) : Lsh[lane * 33 + jj];
            for (int m = 0; m < jj; ++m) sv = fma(-Lsh[lane * 33 + m], Ush[jj * 33 + m], sv);
        }
        const double d = __shfl_sync(0xffffffffu, sv, jj);
        if (!pos_finite(d)) return RS_FIT_NOTPD;
        const double r = rcp_newton(d);
        if (lane == jj) dinv = r;
        else if (act && lane > jj) {
            Lsh[lane * 33 + jj] = sv * r;
            Ush[lane * 33 + jj] = sv;
        }
        __syncwarp();
    }
    double ty = y, t1 = act ? 1.0 : 0.0;
    for (int kk = 0; kk < n; ++kk) {         // L t = rhs, unit diagonal
        const double yk = __shfl_sync(0xffffffffu, ty, kk);
        const double ok = __shfl_sync(0xffffffffu, t1, kk);
        if (act && lane > kk) {
            const double l = Lsh[lane * 33 + kk];
            ty = fma(-l, yk, ty);
            t1 = fma(-l, ok, t1);
        }
    }
    const double sc = act ? t1 * dinv : 0.0;
    double num = act ? sc * ty : 0.0, den = act ? sc * t1 : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    const double b = num * rcp_newton(den);
    double al = act ? fma(-b, t1, ty) * dinv : 0.0;
    for (int kk = n - 1; kk >= 0; --kk) {    // L^T alpha = D^-1 (t_y - b t_1)
        const double ak = __shfl_sync(0xffffffffu, al, kk);
        if (lane < kk) al = fma(-Lsh[kk * 33 + lane], ak, al);
    }
    const int fin = __all_sync(0xffffffffu, !act || finite_bits(al)) && finite_bits(b);
    if (coef) {
        if (act) coef[1 + lane] = al;
        if (lane == 0) coef[0] = b;
    }
    __syncwarp();
    if (!fin) return RS_FIT_NONFINITE;
    if (pt) {                                // predictions, one candidate row per lane
        const int nc = __popcll(pt->cand);
        for (int r0 = 0; r0 < nc; r0 += 32) {
            const bool mine = r0 + lane < nc;
            int t = 0;
            if (mine) t = select_bit(pt->cand, r0 + lane);
            double yh = b;
            for (int q = 0; q < n; ++q) {
                const double aq = __shfl_sync(0xffffffffu, al, q);
                const int vq = __shfl_sync(0xffffffffu, v, q);
                if (mine) yh = fma(aq, __ldg(K + t * RS_GRAM_LD + vq), yh);
            }
            if (mine) {
                const int r = __popcll(pt->test & ((1ull << t) - 1ull));
                if (r < pt->room) pt->dst[r] = yh;
            }
        }
    }
    return RS_FIT_OK;
}

constexpr int kLargeWarps = 4;

// Dynamic shared memory: Lsh [4][32*33] doubles, then without refinement Ush [4][32*33]
// (fit_warp_ldl), with refinement per warp: beta [Fmax], coefficients [64] doubles, pair
// slots [32] ints (fit_warp).
__global__ void __launch_bounds__(kLargeWarps * 32)
solve_large_kernel(const SolveArgs a) {
    __shared__ long long start[kHist], cstart[kHist];
    extern __shared__ __align__(16) double dsm[];
    double* Lall = dsm;
    bucket_tables(a.hist, start, cstart);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* Lsh = Lall + warp * 32 * 33;
    const bool refine = (a.flags & RS_REFINE_X) != 0;
    double* Ush = Lall + (kLargeWarps + warp) * 32 * 33;   // without refinement only
    double* rbase = Lall + kLargeWarps * 32 * 33 + (int64_t)warp * (a.max_feat + 64 + 16);
    const long long first = refine ? start[1] : start[kNMid + 1], end = start[RS_MAXPAIRS + 1];
    for (long long pos = first + (long long)blockIdx.x * kLargeWarps + warp; pos < end;
         pos += (long long)gridDim.x * kLargeWarps) {
        int n = 1;
        while (start[n + 1] <= pos) ++n;
        const uint4 rec = a.recs[pos];
        const int64_t f = rec.x;
        const int64_t s = f / RS_NOPT;
        const int j = (int)(f - s * RS_NOPT);
        const int p = (int)rec.y;
        const double* Kp = a.K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
        const int64_t base = ((int64_t)p * RS_NOPT + j) * RS_MAXPAIRS;
        double* out = coef_out(a, f);
        PredTarget ptv;
        const PredTarget* pt = pred_target(a, s, j, p, ptv) ? &ptv : nullptr;
        RefineCtx rc;
        if (refine) {
            rc.Zp = a.Z + a.x_offsets[p];
            rc.F = a.feat_width[p];
            rc.beta = rbase;
            rc.sh = rbase + a.max_feat;
            rc.vsh = reinterpret_cast<int*>(rbase + a.max_feat + 64);
        }
        const int st = refine ? fit_warp(n, rec.z, a.pb + base, a.ylab + base, Kp, RS_GRAM_LD,
                                         a.lambda, Lsh, out, pt, &rc)
                              : fit_warp_ldl(n, rec.z, a.pb + base, a.ylab + base, Kp,
                                             a.dlam + (int64_t)p * RS_MAXV, Lsh, Ush, out, pt);
        if (lane == 0) {
            if (st != RS_FIT_OK && pt) mark_failed(a, s, j, *pt);
            finish_record(a, f, n, st, out);
        }
        if (a.counters && lane == 0) atomicAdd(a.counters + (st == RS_FIT_OK ? 9 : st == RS_FIT_NOTPD ? 11 : 12), 1ull);
        __syncwarp();
    }
}

// ====================================================================== solve, n > kNMid
// Fits of kNMid < n <= 32 pairs (the leave-one-version-out protocol: 31 pairs per fit), without
// refinement.  kWideLanes lanes share one fit, so a warp works on kWideGroups fits at once.
// The fit's bordered system M = K_TT + lambda I is factored right-looking, M = L D L^T, in a
// packed lower triangle in shared memory: at pivot k every element of the trailing triangle
// takes one FMA, S_ij -= L_ik S_jk, and those elements are spread evenly over the group's
// lanes, so the lanes stay busy as the triangle shrinks (one lane per row would leave half of
// them idle).  The reciprocal of a pivot is one warp instruction for kWideGroups fits.  Then,
// as in solve_fixed: t_y = L^-1 y and t_1 = L^-1 1 (taken in the factorisation's sweep),
// b = t_1^T D^-1 t_y / t_1^T D^-1 t_1, alpha = L^-T D^-1 (t_y - b t_1), predictions
// b + sum_a alpha_a K[t][v_a]
// with the candidate rows spread over the lanes.  Every loop that shuffles runs to the warp's
// largest n, so the groups of a warp (equal n except at bucket boundaries) stay converged.
#ifndef RS_WIDE_LANES
#define RS_WIDE_LANES 16
#endif
constexpr int kWideLanes = RS_WIDE_LANES;                  // lanes per fit: 4, 8, 16 or 32
static_assert(kWideLanes == 4 || kWideLanes == 8 || kWideLanes == 16 || kWideLanes == 32, "lanes per fit");
constexpr int kWideGroups = 32 / kWideLanes;
constexpr int kWideWarps = 2;
constexpr int kWideTri = tri(RS_MAXPAIRS);                 // packed lower triangle with diagonal
constexpr int kWideDoubles = kWideTri + 4 * RS_MAXPAIRS;   // + two pivot columns, t_y, t_1
constexpr size_t kWideSmem = (size_t)kWideWarps * kWideGroups * (kWideDoubles * sizeof(double) +
                                                                 RS_MAXPAIRS * sizeof(int));

// Sum over the kWideLanes lanes of a group (xor offsets stay inside the group).
__device__ __forceinline__ double group_sum(double x) {
#pragma unroll
    for (int o = kWideLanes / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Row and column of entry e of a packed lower triangle (row i holds columns 0..i), and the
// step to entry e + kWideLanes.
__device__ __forceinline__ void tri_pos(int e, int& i, int& j) {
    i = 0;
    while (tri(i + 1) <= e) ++i;
    j = e - tri(i);
}
__device__ __forceinline__ void tri_step(int& i, int& j) {
    j += kWideLanes;
    while (j > i) {
        j -= i + 1;
        ++i;
    }
}

__global__ void __launch_bounds__(kWideWarps * 32)
solve_wide_kernel(const SolveArgs a, unsigned long long* work) {
    __shared__ long long start[kHist], cstart[kHist];
    __shared__ uint16_t tri_rc[tri(RS_MAXPAIRS - 1)];         // packed-triangle entry -> row, column
    extern __shared__ __align__(16) double wsm[];
    for (int i = threadIdx.x >> 5; i < RS_MAXPAIRS - 1; i += kWideWarps)
        for (int j = threadIdx.x & 31; j <= i; j += 32) tri_rc[tri(i) + j] = (uint16_t)(i << 8 | j);
    bucket_tables(a.hist, start, cstart);                      // (ends with a barrier)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / kWideLanes, l = lane % kWideLanes;
    const int gb = warp * kWideGroups + g;                  // fit group of the block
    double* A = wsm + (size_t)gb * kWideDoubles;
    double* C0 = A + kWideTri;
    double* C1 = C0 + RS_MAXPAIRS;
    double* Ty = C1 + RS_MAXPAIRS;
    double* T1 = Ty + RS_MAXPAIRS;
    int* VS = reinterpret_cast<int*>(wsm + (size_t)kWideWarps * kWideGroups * kWideDoubles) + gb * RS_MAXPAIRS;
    const long long lo = start[kNMid + 1], hi = start[RS_MAXPAIRS + 1];
    for (;;) {
        unsigned long long got = 0;
        if (lane == 0) got = atomicAdd(work, (unsigned long long)kWideGroups);
        const long long pos = lo + (long long)__shfl_sync(0xffffffffu, got, 0) + g;
        if (__shfl_sync(0xffffffffu, pos, 0) >= hi) break;
        const bool active = pos < hi;
        int n = 0;
        uint4 rec = make_uint4(0, 0, 0, 0);
        if (active) {
            n = kNMid + 1;
            while (start[n + 1] <= pos) ++n;
            rec = a.recs[pos];
        }
        const int nw = __reduce_max_sync(0xffffffffu, n);
        const int64_t f = rec.x;
        const int64_t s = f / RS_NOPT;
        const int j = (int)(f - s * RS_NOPT);
        const int p = (int)rec.y;
        const double* Kp = a.K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
        const double* dl = a.dlam + (int64_t)p * RS_MAXV;
        const int64_t pbase = ((int64_t)p * RS_NOPT + j) * RS_MAXPAIRS;
        double* out = active ? coef_out(a, f) : nullptr;
        PredTarget ptv;
        const PredTarget* pt = active && pred_target_v(a, s, j, p, (int)rec.w, ptv) ? &ptv : nullptr;
        // the pairs of the fit: slot of the before version, label
        for (int q = l; q < n; q += kWideLanes) {
            const int bit = select_bit(rec.z, q);
            VS[q] = a.pb[pbase + bit];
            Ty[q] = a.ylab[pbase + bit];
            T1[q] = 1.0;
        }
        __syncwarp();
        {                                                    // M, lower triangle
            int i, jj;
            tri_pos(l, i, jj);
            for (int e = l; e < tri(n); e += kWideLanes, tri_step(i, jj))
                A[e] = i == jj ? __ldg(dl + VS[i]) : __ldg(Kp + VS[i] * RS_GRAM_LD + VS[jj]);
        }
        __syncwarp();
        // Right-looking LDL^T with a one-pivot lookahead, and the forward substitution of both
        // right-hand sides folded into the same sweep.  Step k: one lane forms the next pivot
        // d_{k+1} first, so its reciprocal is issued before the trailing update instead of
        // after it; the update of column k+1 also stores that column's L = S / d_{k+1} (and
        // its S for step k+1, in the other pivot-column buffer); the right-hand sides take
        // column k.  One warp barrier per pivot.  From its pivot on, a diagonal slot holds 1/d.
        int st = active ? RS_FIT_OK : RS_FIT_EMPTY;
        {
            const bool kin = n > 0;
            const double d = kin ? A[0] : 1.0;
            if (kin && !pos_finite(d)) st = RS_FIT_NOTPD;
            const bool go = kin && st == RS_FIT_OK;
            const double r = rcp_newton(go ? d : 1.0);
            if (go)
                for (int i = 1 + l; i < n; i += kWideLanes) {
                    const double c = A[tri(i)];
                    C0[i] = c;
                    A[tri(i)] = c * r;
                }
            __syncwarp();
            if (go && l == 0) A[0] = r;
        }
        for (int k = 0; k + 1 < nw; ++k) {
            const bool kin = k + 1 < n && st == RS_FIT_OK;
            const double* Ck = (k & 1) ? C1 : C0;
            double* Cn = (k & 1) ? C0 : C1;
            double dn = 1.0;                                 // S_{k+1,k+1} - L_{k+1,k} S_{k+1,k}
            if (kin && l == 0) dn = fma(-A[tri(k + 1) + k], Ck[k + 1], A[tri(k + 1) + k + 1]);
            dn = __shfl_sync(0xffffffffu, dn, g * kWideLanes);
            if (kin && !pos_finite(dn)) st = RS_FIT_NOTPD;
            const bool go = kin && st == RS_FIT_OK;
            const double rn = rcp_newton(go ? dn : 1.0);
            if (go) {
                // the work items of the step, dealt to the group's lanes round-robin across
                // the three loops (o: the lane that takes a loop's first item)
                const int m = n - k - 1;
                int o = 0;
                for (int ri = k + 2 + ((l - o) & (kWideLanes - 1)); ri < n; ri += kWideLanes) {
                    const double v = fma(-A[tri(ri) + k], Ck[k + 1], A[tri(ri) + k + 1]);
                    Cn[ri] = v;                              // column k+1: S for step k+1,
                    A[tri(ri) + k + 1] = v * rn;             // L = S / d_{k+1}
                }
                o = (o + m - 1) & (kWideLanes - 1);
                {                                            // rows and columns > k+1
                    const int T = tri(m - 1);
#pragma unroll 4
                    for (int e = (l - o) & (kWideLanes - 1); e < T; e += kWideLanes) {
                        const int ij = tri_rc[e];            // row << 8 | column of entry e
                        const int ri = k + 2 + (ij >> 8), cj = k + 2 + (ij & 255);
                        A[tri(ri) + cj] = fma(-A[tri(ri) + k], Ck[cj], A[tri(ri) + cj]);
                    }
                }
                o = (o + tri(m - 1)) & (kWideLanes - 1);
                const double yk = Ty[k], ok1 = T1[k];        // t -= L_{.,k} t_k
                for (int ri = k + 1 + ((l - o) & (kWideLanes - 1)); ri < n; ri += kWideLanes) {
                    const double L = A[tri(ri) + k];
                    Ty[ri] = fma(-L, yk, Ty[ri]);
                    T1[ri] = fma(-L, ok1, T1[ri]);
                }
                if (l == 0) A[tri(k + 1) + k + 1] = rn;
            }
            __syncwarp();
        }
        const bool ok = active && st == RS_FIT_OK;
        double num = 0.0, den = 0.0;
        if (ok)
            for (int i = l; i < n; i += kWideLanes) {
                const double sc = T1[i] * A[tri(i) + i];
                num = fma(sc, Ty[i], num);
                den = fma(sc, T1[i], den);
            }
        num = group_sum(num);
        den = group_sum(den);
        const double b = num * rcp_newton(ok ? den : 1.0);
        if (ok)
            for (int i = l; i < n; i += kWideLanes) Ty[i] = fma(-b, T1[i], Ty[i]) * A[tri(i) + i];
        __syncwarp();
        for (int k = nw - 1; k >= 0; --k) {                  // L^T alpha = D^-1 (t_y - b t_1)
            if (ok && k < n) {
                const double ak = Ty[k];
                for (int i = l; i < k; i += kWideLanes) Ty[i] = fma(-A[tri(k) + i], ak, Ty[i]);
            }
            __syncwarp();
        }
        bool bad = ok && !finite_bits(b);
        if (ok)
            for (int i = l; i < n; i += kWideLanes) bad = bad || !finite_bits(Ty[i]);
        const unsigned gm = kWideLanes == 32 ? 0xffffffffu : ((1u << (kWideLanes & 31)) - 1u) << (g * kWideLanes);
        const unsigned badm = __ballot_sync(0xffffffffu, bad);
        if (ok && (badm & gm)) st = RS_FIT_NONFINITE;
        if (out && st == RS_FIT_OK) {
            if (l == 0) out[0] = b;
            for (int i = l; i < n; i += kWideLanes) out[1 + i] = Ty[i];
        }
        // predictions b + sum_a alpha_a K[t][v_a], summed in pair order like every other
        // solver; the group's lanes take the candidate rows in turn
        if (pt && st == RS_FIT_OK) {
            int c = 0;
            for (uint64_t cm = pt->cand; cm; cm &= cm - 1, ++c) {
                if (c % kWideLanes != l) continue;
                const int t = __ffsll((long long)cm) - 1;
                const double* Kt = Kp + t * RS_GRAM_LD;
                double yh = b;
                for (int q = 0; q < n; ++q) yh = fma(Ty[q], __ldg(Kt + VS[q]), yh);
                const int r = __popcll(pt->test & ((1ull << t) - 1ull));
                if (r < pt->room) pt->dst[r] = yh;
            }
        }
        if (active && l == 0) {
            if (st != RS_FIT_OK && pt) mark_failed(a, s, j, *pt);
            finish_record(a, f, n, st, out);
        }
        count_status(a, st, active && l == 0);
        __syncwarp();
    }
}

// ====================================================================== closed-form leave-one-out
// RS_LOO_CLOSED.  A split that holds out one version removes, for optimization j, at most the
// one pair of the program's pairs for j that contains that version (a version is the before
// or the after side of at most one pair per j).  The fit's system is then the program's full
// M = K_PP + lambda I for j without row and column i, and with w_y = M^-1 y, w_1 = M^-1 1 and
// u = row i of the symmetric M^-1, deleting index i from a linear system gives, for q != i,
//   (M_r^-1 y)_q = w_y[q] - u_q w_y[i] / u_i,     (M_r^-1 1)_q = w_1[q] - u_q w_1[i] / u_i.
// b and alpha then follow as in every solver (Sec. 3.4): b = sum t_y / sum t_1 and
// alpha = t_y - b t_1.  One inverse per (program, j) replaces a factorization per fit.
// the table of one (program, optimization): M^-1 (32 x 32, row-major), w_y, w_1, then the
// sums 1^T w_y and 1^T w_1 (padded to a 32-byte multiple)
constexpr int kLooWy = RS_MAXPAIRS * RS_MAXPAIRS;
constexpr int kLooW1 = kLooWy + RS_MAXPAIRS;
constexpr int kLooSum = kLooW1 + RS_MAXPAIRS;
constexpr int kLooTab = kLooSum + 4;                                   // doubles per (p, j)
constexpr int kLooFitThreads = 256;

// One warp per (program, optimization): Gauss-Jordan elimination of [M | y | 1] without
// pivoting (M is symmetric positive definite), lane i holding row i in registers, padded
// with the identity past n (inert: a padded row or column meets only zeros), so that every
// index is static.  Step k: every row i != k subtracts A_ik / p_k times row k (p_k = A_kk,
// the pivot; row k reaches the others through shared memory) and stores -A_ik / p_k in
// column k, the right block's column that column k's elimination has made; row k stays and
// stores 1 there.  The left block ends diagonal, diag(p), so M^-1 is each row of the right
// block divided by its pivot.  Row k needs no scaling inside the loop, so every lane runs the
// same instructions.  Writes the symmetrized inverse, w_y, w_1 and their sums to tab, and
// ok = 1 when every pivot was positive and finite.  A non-finite label enters y as 0 and sets
// its pair's bit in bad: a fit that trains on that pair is non-finite, and one that leaves it
// out does not depend on its label (the deletion formula above holds for any value in
// position i).
__global__ void __launch_bounds__(32)
loo_inv_kernel(const int64_t* __restrict__ row_off, const double* __restrict__ K,
               const uint8_t* __restrict__ pb, const double* __restrict__ ylab,
               const int* __restrict__ npair, const double* __restrict__ dlam, double* tab, uint8_t* ok,
               uint32_t* bad) {
    __shared__ __align__(16) double rowk[RS_MAXPAIRS + 2];     // the pivot row and its right-hand sides
    __shared__ double S[RS_MAXPAIRS][RS_MAXPAIRS + 1];          // the inverse, for the symmetrized store
    __shared__ int vs[RS_MAXPAIRS];
    const int pj = blockIdx.x, p = pj / RS_NOPT, i = threadIdx.x;
    const int V = (int)(row_off[p + 1] - row_off[p]);
    const int n = V >= 1 && V <= RS_MAXV ? npair[pj] : 0;
    if (n < 1 || n > RS_MAXPAIRS) {
        if (i == 0) {
            ok[pj] = 0;
            bad[pj] = 0;
        }
        return;
    }
    const double* Kp = K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
    const bool row = i < n;
    if (row) vs[i] = pb[(int64_t)pj * RS_MAXPAIRS + i];
    __syncwarp();
    double A[RS_MAXPAIRS], y = 0.0, one = 0.0;
    const int vi = row ? vs[i] : 0;
#pragma unroll
    for (int c = 0; c < RS_MAXPAIRS; ++c) {
        double v = c == i ? 1.0 : 0.0;
        if (row && c < n) v = c == i ? dlam[(int64_t)p * RS_MAXV + vi] : __ldg(Kp + vi * RS_GRAM_LD + vs[c]);
        A[c] = v;
    }
    if (row) {
        y = ylab[(int64_t)pj * RS_MAXPAIRS + i];
        one = 1.0;
    }
    const bool yb = row && !finite_bits(y);
    const unsigned badm = __ballot_sync(0xffffffffu, yb);
    if (yb) y = 0.0;
    double piv = 1.0;                                           // this row's pivot
    bool good = true;
#pragma unroll
    for (int k = 0; k < RS_MAXPAIRS; ++k) {
        if (i == k) {
#pragma unroll
            for (int c = 0; c < RS_MAXPAIRS; c += 2)
                *reinterpret_cast<double2*>(rowk + c) = make_double2(A[c], A[c + 1]);
            rowk[RS_MAXPAIRS] = y;
            rowk[RS_MAXPAIRS + 1] = one;
        }
        __syncwarp();
        const double d = rowk[k];                               // the same value in every lane
        good = good && pos_finite(d);
        const double r = rcp_newton(good ? d : 1.0);
        const double fr = i == k ? 0.0 : A[k] * r;
        if (i == k) piv = d;
#pragma unroll
        for (int c = 0; c < RS_MAXPAIRS; c += 2) {
            const double2 rk = *reinterpret_cast<const double2*>(rowk + c);
            if (c != k) A[c] = fma(-fr, rk.x, A[c]);
            if (c + 1 != k) A[c + 1] = fma(-fr, rk.y, A[c + 1]);
        }
        y = fma(-fr, rowk[RS_MAXPAIRS], y);
        one = fma(-fr, rowk[RS_MAXPAIRS + 1], one);
        A[k] = i == k ? 1.0 : -fr;
        __syncwarp();                                           // before the next pivot row
    }
    if (good) {
        const double rp = rcp_newton(piv);
#pragma unroll
        for (int c = 0; c < RS_MAXPAIRS; ++c) S[i][c] = A[c] * rp;
        y *= rp;
        one *= rp;
        __syncwarp();
        double* T = tab + (int64_t)pj * kLooTab;
        for (int rr = 0; rr < n; ++rr)
            if (row) T[rr * RS_MAXPAIRS + i] = 0.5 * (S[rr][i] + S[i][rr]);
        if (row) {
            T[kLooWy + i] = y;
            T[kLooW1 + i] = one;
        }
        const double sy = warp_sum(y), s1 = warp_sum(one);    // lanes past n hold 0
        if (i == 0) {
            T[kLooSum] = sy;
            T[kLooSum + 1] = s1;
        }
    }
    if (i == 0) {
        ok[pj] = good ? 1 : 0;
        bad[pj] = badm;
    }
}

// One thread per fit.  With u_i = (M^-1)_ii and 1^T u = w_1[i] (M^-1 is symmetric), deleting
// pair i turns the sums that give b into one-term downdates,
//   1^T t_y = 1^T w_y - w_1[i] w_y[i] / u_i,     1^T t_1 = 1^T w_1 - w_1[i]^2 / u_i,
// so b = 1^T t_y / 1^T t_1 costs O(1), and alpha_q = (w_y[q] - b w_1[q]) - u_q e for q != i,
// e = (w_y[i] - b w_1[i]) / u_i.  The prediction at pair i's own before version v_i -- the
// held-out version whenever it lacks j -- needs no sum either: with K_PP = M - lambda I,
//   b + sum_{q != i} alpha_q K[v_i][v_q] = y_i - e
// (the leave-one-out residual of kernel ridge, with the intercept refitted; y_i the value that
// entered the inverse).  Other candidate rows (a version without a partner for j, or the
// after versions that RS_RANK_ALL ranks) take the sum over the fit's pairs in pair order, as
// the direct solvers do.  A fit whose training pairs lack more than one of its program's pairs
// for j has no closed form here: RS_EDATA (detail: the program), and the fit is reported
// failed.  Non-finite b or e: RS_FIT_NONFINITE.  Fits without a pair were finished by the
// bucket pass.
__global__ void __launch_bounds__(kLooFitThreads)
loo_fit_kernel(const SolveArgs a, int64_t S6, const int* __restrict__ npair,
               const double* __restrict__ tab, const uint8_t* __restrict__ tab_ok,
               const uint32_t* __restrict__ tab_bad) {
    const int64_t f = (int64_t)blockIdx.x * kLooFitThreads + threadIdx.x;
    const int n = f < S6 ? a.fit_key[f] / kCntBins : 0;
    const bool active = n > 0;
    int st = RS_FIT_EMPTY;
    if (active) {
        const int64_t s = f / RS_NOPT;
        const int j = (int)(f - s * RS_NOPT);
        const int p = a.split_prog[s];
        const int pj = p * RS_NOPT + j;
        const int N = npair[pj];
        const uint32_t pm = a.fit_pm[f];
        const uint32_t full = N >= 32 ? 0xffffffffu : (1u << N) - 1u;
        const uint32_t removed = full & ~pm;
        const double* T = tab + (int64_t)pj * kLooTab;
        st = RS_FIT_OK;
        if (__popc(removed) > 1 || (pm & ~full)) {
            st = RS_FIT_NOTPD;
            rs_dev_flag(a.dstatus, RS_EDATA, p);
        } else if (!tab_ok[pj]) {
            st = RS_FIT_NOTPD;
        } else if (pm & tab_bad[pj]) {
            st = RS_FIT_NONFINITE;           // a label of the fit's pairs is not finite
        }
        const int i = removed ? __ffs(removed) - 1 : -1;
        double b = 0.0, e = 0.0;
        if (st == RS_FIT_OK) {
            double num = T[kLooSum], den = T[kLooSum + 1], cy = 0.0, c1 = 0.0;
            if (i >= 0) {
                const double ui = T[i * RS_MAXPAIRS + i];
                if (!pos_finite(ui)) {
                    st = RS_FIT_NOTPD;
                } else {
                    const double ri = rcp_newton(ui), wyi = T[kLooWy + i], w1i = T[kLooW1 + i];
                    cy = wyi * ri;
                    c1 = w1i * ri;
                    num = fma(-w1i, cy, num);
                    den = fma(-w1i, c1, den);
                }
            }
            if (st == RS_FIT_OK) {
                b = num * rcp_newton(den);
                e = fma(-b, c1, cy);
                if (!finite_bits(b) || !finite_bits(e)) st = RS_FIT_NONFINITE;
            }
        }
        const uint8_t* pbj = a.pb + (int64_t)pj * RS_MAXPAIRS;
        auto alpha = [&](int q) {
            const double al = fma(-b, T[kLooW1 + q], T[kLooWy + q]);
            return i >= 0 ? fma(-T[i * RS_MAXPAIRS + q], e, al) : al;
        };
        double* out = a.coef_user ? a.coef + f * RS_COEF_STRIDE : nullptr;   // no compact records
        if (out && st == RS_FIT_OK) {
            out[0] = b;
            int c = 1;
            for (uint32_t m = pm; m; m &= m - 1) out[c++] = alpha(__ffs(m) - 1);
        }
        PredTarget pt;
        const bool has = pred_target_v(a, s, j, p, (int)(a.row_off[p + 1] - a.row_off[p]), pt);
        if (has && st == RS_FIT_OK) {
            const int vi = i >= 0 ? pbj[i] : -1;
            const double* Kp = a.K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
            for (uint64_t cm = pt.cand; cm; cm &= cm - 1) {
                const int t = __ffsll((long long)cm) - 1;
                double yh;
                if (t == vi) {
                    const double yi = a.ylab[(int64_t)pj * RS_MAXPAIRS + i];
                    yh = (finite_bits(yi) ? yi : 0.0) - e;
                } else {
                    yh = b;
                    for (uint32_t m = pm; m; m &= m - 1) {
                        const int q = __ffs(m) - 1;
                        yh = fma(alpha(q), __ldg(Kp + t * RS_GRAM_LD + pbj[q]), yh);
                    }
                }
                const int r = __popcll(pt.test & ((1ull << t) - 1ull));
                if (r < pt.room) pt.dst[r] = yh;
            }
        }
        if (st != RS_FIT_OK && has) mark_failed(a, s, j, pt);
        finish_record(a, f, n, st, out);
    }
    count_status(a, st, active);
}

// ====================================================================== rank pass
// One thread per test row: its row record and its six predictions (written by the solve
// kernels) go through rank_row; no FP64 arithmetic.
#ifndef RS_RANK_TILE
#define RS_RANK_TILE 256
#endif
#ifndef RS_RANK_MINB
#define RS_RANK_MINB 3
#endif
constexpr int kRankTile = RS_RANK_TILE;      // rows per tile (one ring stage) = consumer threads
constexpr int kRankWarps = kRankTile / 32;   // consumer warps
constexpr int kRankThreads = kRankTile + 32; // and one producer warp
constexpr int kRankStages = 3;
constexpr int kRankPlanes = 1 + RS_NOPT;     // the row records, then the six prediction planes
constexpr size_t kRankStageBytes = (size_t)kRankPlanes * kRankTile * 8;
constexpr size_t kRankOutBytes = (size_t)kRankTile * 3 * 8;   // a warp's top-3 values, per warp
constexpr size_t kRankSmem = kRankStages * kRankStageBytes + 2 * kRankStages * 8 + kRankOutBytes;
static_assert(kRankTile % 32 == 0, "whole warps of rows");

// Persistent blocks over tiles of kRankTile rows, a producer warp and kRankWarps consumer
// warps that never wait for one another.  The producer's lane 0 streams each tile -- the row
// records and the six prediction planes, seven 1-D TMA bulk copies -- into a 3-stage
// shared-memory ring: a stage is refilled once every consumer warp has arrived on its "empty"
// mbarrier, and its copies complete on its "full" mbarrier.  A consumer warp waits for the
// stage, reads its 32 rows into registers (one per lane), arrives on
// "empty" and ranks the rows while the copies of the tiles ahead fly.  The reported values of a
// warp's 32 rows (32 k doubles, contiguous in rec_pred) are gathered in shared memory and
// written as 16-byte stores, instead of each lane's k scattered 8-byte stores.  Bounded waits:
// on a timeout RS_ETIMEOUT is set and the warp leaves; the producer waits (bounded) for the
// copies it has in flight before it leaves.
template <bool PACK>
__global__ void __launch_bounds__(kRankThreads, RS_RANK_MINB)
rank_pass_kernel(const RankPassArgs a) {
    extern __shared__ __align__(128) unsigned char rsm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t total = a.rec_offsets[a.S];
    const int64_t nrows = total < a.R ? total : a.R;
    if (total > a.R && blockIdx.x == 0 && tid == 0) rs_dev_flag(a.dstatus, RS_EDATA, -3);
    const int64_t ntiles = (nrows + kRankTile - 1) / kRankTile;
    const uint32_t sbase = tc::smem_u32(rsm);
    const uint32_t full0 = sbase + (uint32_t)(kRankStages * kRankStageBytes);
    const uint32_t empty0 = full0 + 8 * kRankStages;
    if (tid == 0) {
        for (int st = 0; st < kRankStages; ++st) {
            tc::mbar_init(full0 + 8 * st, 1);
            tc::mbar_init(empty0 + 8 * st, kRankWarps);
        }
        tc::fence_barrier_init();
    }
    __syncthreads();
    if (warp == kRankWarps) {                  // producer
        if (lane != 0) return;
        int64_t q = 0;                         // tiles issued
        int st = 0;
        uint32_t eph = 0;                      // parity of the next "empty" phase to wait for
        bool failed = false;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++q) {
            if (q >= kRankStages &&            // every consumer warp has read the stage's last tile
                !tc::mbar_wait(empty0 + 8 * st, eph, a.dstatus, -22)) {
                failed = true;
                break;
            }
            tc::fence_proxy_async_smem();
            const int64_t row0 = tile * kRankTile;
            const int64_t rows = nrows - row0 < kRankTile ? nrows - row0 : kRankTile;
            // even: a 16-byte multiple (stays inside the buffers: PS and the record array are even)
            const uint32_t bytes = (uint32_t)((rows + 1) & ~(int64_t)1) * 8;
            const uint32_t bar = full0 + 8 * st;
            const uint32_t dst = sbase + (uint32_t)(st * kRankStageBytes);
            tc::mbar_expect_tx(bar, bytes * kRankPlanes);
            tc::bulk_load(dst, a.row_info + row0, bytes, bar);
#pragma unroll
            for (int j = 0; j < RS_NOPT; ++j)
                tc::bulk_load(dst + (uint32_t)((1 + j) * kRankTile * 8), a.predbuf + (int64_t)j * a.PS + row0, bytes, bar);
            if (++st == kRankStages) {
                st = 0;
                if (q >= kRankStages) eph ^= 1u;
            }
        }
        if (failed)                            // the copies of tiles q - 3 .. q - 1 were issued
            for (int64_t x = q - 1; x >= 0 && x >= q - kRankStages; --x)
                tc::mbar_wait(full0 + 8 * (int)(x % kRankStages), (uint32_t)((x / kRankStages) & 1), a.dstatus, -23);
        return;
    }
    RankTally c;
    int st = 0;
    uint32_t par = 0;
    // this warp's slots for the reported values: [32 rows][3]
    double* wout = reinterpret_cast<double*>(rsm + kRankStages * kRankStageBytes + 2 * kRankStages * 8) +
                   (size_t)warp * 32 * 3;
    // k = 3 (the method's top-3) with a 16-byte aligned rec_pred; other k store per lane
    const bool stage_out = !PACK && a.rec_pred && a.k == 3 && (reinterpret_cast<uintptr_t>(a.rec_pred) & 15) == 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const bool ok = tc::mbar_wait(full0 + 8 * st, par, a.dstatus, -20);
        if (!__all_sync(0xffffffffu, ok)) return;
        const unsigned char* stage = rsm + st * kRankStageBytes;
        const int64_t row = tile * kRankTile + tid;
        const bool in = row < nrows;
        const unsigned long long info = in ? reinterpret_cast<const unsigned long long*>(stage)[tid] : 0ull;
        double pred[RS_NOPT];
#pragma unroll
        for (int j = 0; j < RS_NOPT; ++j)
            pred[j] = in ? reinterpret_cast<const double*>(stage + (1 + j) * kRankTile * 8)[tid] : 0.0;
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(empty0 + 8 * st);   // this warp has read the stage
        if (++st == kRankStages) {
            st = 0;
            par ^= 1u;
        }
        if constexpr (PACK) {                  // the tile's recommendations, for the packed output
            const int nrec = in ? rank_row<true>(a, row, info, pred, c) : 0;
            const unsigned v = __reduce_add_sync(0xffffffffu, (unsigned)nrec);
            if (lane == 0 && v) atomicAdd(a.tile_sum + tile, (unsigned long long)v);
        } else if (stage_out) {
            if (in) rank_row<false, true, 3>(a, row, info, pred, c, wout + lane * 3);
            __syncwarp();
            // the warp's 32 rows: 96 contiguous doubles of rec_pred
            const int64_t wrow = tile * kRankTile + warp * 32;
            const double2* src = reinterpret_cast<const double2*>(wout);
            double2* dst = reinterpret_cast<double2*>(a.rec_pred + wrow * 3);
            if (wrow + 32 <= nrows) {                  // a whole warp of rows: 48 pairs
                dst[lane] = src[lane];
                if (lane < 16) dst[32 + lane] = src[32 + lane];
            } else {
                const int64_t nv = (nrows - wrow) * 3;               // doubles (none past the end)
                const double* s1 = reinterpret_cast<const double*>(src);
                double* d1 = reinterpret_cast<double*>(dst);
                for (int64_t q = lane; q < nv; q += 32) d1[q] = s1[q];
            }
            __syncwarp();
        } else {
            if (in) rank_row(a, row, info, pred, c);
        }
    }
    if (a.counters) {
        const uint32_t vals[10] = {c.rows, c.pred, c.scored, c.sign, c.rec, c.reck, c.rech, c.t1, c.t1h, c.inv};
        const int slot[10] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 13};
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            const uint32_t v = __reduce_add_sync(0xffffffffu, vals[q]);
            if (lane == 0 && v) atomicAdd(a.counters + slot[q], (unsigned long long)v);
        }
    }
}

// ====================================================================== packed predictions
// RS_PACK_PRED: row r's c_r reported predictions go to rec_pred[P_r .. P_r + c_r - 1] with
// P_r = sum of c over the rows before r.  The rank pass leaves each row's list in its plane
// slots and the per-tile totals; tile_scan_kernel turns the totals into tile offsets (one
// block: contiguous chunks per thread, then a block scan), pack_pred_kernel scans the counts
// of each tile's rows (from rec_code) and writes the lists in place.
constexpr int kScanThreads = 1024;

constexpr int kScanItems = 8;                // tiles per thread and round (64 contiguous bytes)

// Exclusive scan of the tiles' recommendation counts, one block: rounds of 8192 tiles, each
// thread loading its 8 consecutive counts as 16-byte vectors, a block scan of the threads'
// sums, and the running total of the earlier rounds carried along.
__global__ void __launch_bounds__(kScanThreads)
tile_scan_kernel(const unsigned long long* __restrict__ tile_sum, unsigned long long* __restrict__ tile_off,
                 int64_t ntiles) {
    __shared__ unsigned long long wsum[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long carry = 0;
    for (int64_t base = 0; base < ntiles; base += (int64_t)kScanThreads * kScanItems) {
        const int64_t i0 = base + (int64_t)tid * kScanItems;
        const bool whole = i0 + kScanItems <= ntiles;
        unsigned long long v[kScanItems];
        if (whole) {
#pragma unroll
            for (int q = 0; q < kScanItems / 2; ++q) {
                const ulonglong2 x = reinterpret_cast<const ulonglong2*>(tile_sum + i0)[q];
                v[2 * q] = x.x;
                v[2 * q + 1] = x.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kScanItems; ++k) v[k] = i0 + k < ntiles ? tile_sum[i0 + k] : 0ull;
        }
        unsigned long long s = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) s += v[k];
        unsigned long long incl = s;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = wsum[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        unsigned long long off = carry + incl - s + (warp > 0 ? wsum[warp - 1] : 0ull);
        unsigned long long o[kScanItems];
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            o[k] = off;
            off += v[k];
        }
        if (whole) {
#pragma unroll
            for (int q = 0; q < kScanItems / 2; ++q)
                reinterpret_cast<ulonglong2*>(tile_off + i0)[q] = make_ulonglong2(o[2 * q], o[2 * q + 1]);
        } else {
#pragma unroll
            for (int k = 0; k < kScanItems; ++k)
                if (i0 + k < ntiles) tile_off[i0 + k] = o[k];
        }
        carry += wsum[kScanThreads / 32 - 1];
        __syncthreads();                     // wsum is written again in the next round
    }
}

__global__ void __launch_bounds__(kRankTile)
pack_pred_kernel(const int64_t* __restrict__ rec_offsets, int64_t S, int64_t R, const uint32_t* __restrict__ rec_code,
                 const double* __restrict__ planes, int64_t PS, const unsigned long long* __restrict__ tile_off,
                 double* __restrict__ out) {
    __shared__ unsigned wsum[kRankTile / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t total = rec_offsets[S];
    const int64_t nrows = total < R ? total : R;
    const int64_t tile = blockIdx.x;
    if (tile * kRankTile >= nrows) return;
    const int64_t row = tile * kRankTile + tid;
    const unsigned c = row < nrows ? (rec_code[row] & 0xFu) : 0u;
    // the row's parked values and the tile's offset are loaded before the block's scan, so
    // their latency overlaps it
    const unsigned long long toff = tile_off[tile];
    double val[RS_NOPT];
#pragma unroll
    for (int pos = 0; pos < RS_NOPT; ++pos) val[pos] = pos < (int)c ? planes[pos * PS + row] : 0.0;
    unsigned incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    unsigned before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    const unsigned long long off = toff + before + (incl - c);
#pragma unroll
    for (int pos = 0; pos < RS_NOPT; ++pos)
        if (pos < (int)c) out[off + pos] = val[pos];
}

// ====================================================================== predict / rank (chunked)
template <int WARPS, bool FIT>
struct RankSmem {
    static constexpr int kPool = FIT ? 32 * 33 : 1;
    double K[RS_MAXV * kKld];
    double lt[RS_MAXV];
    double ylab[RS_NOPT][RS_MAXPAIRS];
    double coef[kFits][RS_COEF_STRIDE];
    double pool[WARPS][kPool];
    long long act_key[RS_MAXV][RS_NOPT];
    uint64_t tmask[kChunk];
    uint32_t pmask[kFits];
    int row_base[kChunk + 1];
    int npair[RS_NOPT];
    uint8_t nfit[kFits];
    uint8_t status[kFits];
    uint8_t known[RS_MAXV];
    uint8_t pair_b[RS_NOPT][RS_MAXPAIRS];
    uint8_t msk[RS_MAXV];
    int8_t slot_of[RS_MAXV];
    int cur_prog, V, item, prog_ok;
};

// FIT = true: the plain form, every fit solved here by one warp.  FIT = false: the
// coefficients come from coef_in (compact records at coef_off, or the caller's
// [S][6][33] layout) and the statuses from status_in (or from whether b is finite).
template <int WARPS, bool FIT>
__global__ void __launch_bounds__(WARPS * 32, FIT ? 1 : 2)
rank_kernel(const rs_fit_args a, const int64_t* __restrict__ coef_off,
            const uint8_t* __restrict__ status_in) {
    using Sm = RankSmem<WARPS, FIT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm& sm = *reinterpret_cast<Sm*>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NT = WARPS * 32;
    const int64_t n_items = (a.S + kChunk - 1) / kChunk;
    uint32_t cnt[RS_NCOUNTERS];
#pragma unroll
    for (int c = 0; c < RS_NCOUNTERS; ++c) cnt[c] = 0;
    const long long ktau = okey(a.log_tau);

    if (tid == 0) sm.cur_prog = -1;
    for (;;) {
        __syncthreads();
        if (tid == 0) sm.item = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int64_t item = sm.item;
        if (item >= n_items) break;
        int64_t s0 = item * kChunk;
        const int64_t s1 = min(s0 + (int64_t)kChunk, a.S);
        while (s0 < s1) {
            const int p = rs_find_segment(a.split_offsets, a.P, s0);
            const int64_t seg_end = min(s1, a.split_offsets[p + 1]);
            const int ns = (int)(seg_end - s0);
            // ---------------------------------------------------------- stage program p
            if (p != sm.cur_prog) {
                __syncthreads();
                const int64_t r0 = a.row_offsets[p];
                const int V = (int)(a.row_offsets[p + 1] - r0);
                const bool ok = V >= 1 && V <= RS_MAXV;
                if (!ok && tid == 0) rs_dev_flag(a.dstatus, RS_EDATA, p);
                if (ok) {
                    const double* Kg = a.K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
                    for (int e = tid; e < V * RS_MAXV; e += NT) {
                        const int r = e >> 6, c = e & 63;
                        sm.K[r * kKld + c] = (c < V) ? Kg[e] : 0.0;
                    }
                    for (int r = tid; r < RS_MAXV; r += NT) {
                        sm.slot_of[r] = -1;
                        if (r < V) {
                            sm.lt[r] = a.log_time[r0 + r];
                            sm.msk[r] = a.masks[r0 + r] & 63;
                        }
                    }
                }
                __syncthreads();
                if (ok && tid < V) sm.slot_of[sm.msk[tid]] = (int8_t)tid;
                __syncthreads();
                if (ok && tid < RS_NOPT) {
                    const int j = tid;
                    int np = 0;
                    for (int v = 0; v < V; ++v) {
                        const int m = sm.msk[v];
                        if ((m >> j) & 1) continue;
                        const int w = sm.slot_of[m | (1 << j)];
                        if (w < 0) continue;
                        if (np == RS_MAXPAIRS) {      // only possible with repeated masks
                            rs_dev_flag(a.dstatus, RS_EDATA, p);
                            break;
                        }
                        sm.pair_b[j][np] = (uint8_t)v;
                        sm.ylab[j][np] = sm.lt[v] - sm.lt[w];
                        ++np;
                    }
                    sm.npair[j] = np;
                }
                // actual log speedups of adding j to each version, as order keys
                if (ok && tid < V) {
                    const int m = sm.msk[tid];
                    uint8_t kn = 0;
                    for (int j = 0; j < RS_NOPT; ++j) {
                        const int w = ((m >> j) & 1) ? -1 : sm.slot_of[m | (1 << j)];
                        long long key = 0;
                        if (w >= 0) {
                            key = okey(sm.lt[tid] - sm.lt[w]);
                            kn |= (uint8_t)(1u << j);
                        }
                        sm.act_key[tid][j] = key;
                    }
                    sm.known[tid] = kn;
                }
                if (tid == 0) {
                    sm.cur_prog = p;
                    sm.V = V;
                    sm.prog_ok = ok;
                }
                __syncthreads();
            }
            const int V = sm.V;
            if (!sm.prog_ok) {
                s0 = seg_end;
                continue;
            }
            const uint64_t full = rs_full_mask(V);
            // ---------------------------------------------------------- fits of the chunk
            for (int i = tid; i < ns; i += NT) sm.tmask[i] = a.train_masks[s0 + i] & full;
            __syncthreads();
            for (int f = tid; f < ns * RS_NOPT; f += NT) {
                const int i = f / RS_NOPT, j = f % RS_NOPT;
                const uint64_t T = sm.tmask[i];
                uint32_t pm = 0;
                for (int q = 0; q < sm.npair[j]; ++q) {
                    const int v = sm.pair_b[j][q];
                    const int w = sm.slot_of[sm.msk[v] | (1 << j)];
                    if (((T >> v) & 1) && ((T >> w) & 1)) pm |= 1u << q;
                }
                sm.pmask[f] = pm;
                const int n = __popc(pm);
                sm.nfit[f] = (uint8_t)n;
                if (!FIT) {
                    const int64_t gf = s0 * RS_NOPT + f;
                    const double* src = a.coef_in + (coef_off ? coef_off[gf] : gf * RS_COEF_STRIDE);
                    int st;
                    if (status_in) st = status_in[gf];
                    else st = (n > 0 && finite_bits(src[0])) ? RS_FIT_OK : RS_FIT_EMPTY;
                    sm.status[f] = (uint8_t)st;
                    if (st == RS_FIT_OK)
                        for (int e = 0; e <= n; ++e) sm.coef[f][e] = src[e];
                } else if (n == 0) {
                    sm.status[f] = RS_FIT_EMPTY;
                }
            }
            __syncthreads();
            if (FIT) {
                for (int f = warp; f < ns * RS_NOPT; f += WARPS) {
                    const int n = sm.nfit[f];
                    if (n == 0) continue;
                    const int j = f % RS_NOPT;
                    const int st = fit_warp(n, sm.pmask[f], sm.pair_b[j], sm.ylab[j], sm.K, kKld,
                                            a.lambda, sm.pool[warp], sm.coef[f]);
                    if (lane == 0) sm.status[f] = (uint8_t)st;
                    __syncwarp();
                }
                __syncthreads();
                for (int f = tid; f < ns * RS_NOPT; f += NT) {
                    const int st = sm.status[f];
                    cnt[9] += st == RS_FIT_OK;
                    cnt[10] += st == RS_FIT_EMPTY;
                    cnt[11] += st == RS_FIT_NOTPD;
                    cnt[12] += st == RS_FIT_NONFINITE;
                }
                if (a.coef_out) {
                    double* dst = a.coef_out + s0 * RS_NOPT * (int64_t)RS_COEF_STRIDE;
                    for (int e = tid; e < ns * RS_NOPT * RS_COEF_STRIDE; e += NT) {
                        const int f = e / RS_COEF_STRIDE, c = e % RS_COEF_STRIDE;
                        const bool ok = sm.status[f] == RS_FIT_OK;
                        double v = ok ? sm.coef[f][c] : (c == 0 ? nan_d() : 0.0);
                        if (c > sm.nfit[f]) v = 0.0;
                        dst[e] = v;
                    }
                }
                if (a.status_out)
                    for (int f = tid; f < ns * RS_NOPT; f += NT) a.status_out[s0 * RS_NOPT + f] = sm.status[f];
            }
            // ---------------------------------------------------------- predict, rank, score
            if (a.rec_code) {
                if (tid == 0) {
                    int acc = 0;
                    for (int i = 0; i < ns; ++i) {
                        sm.row_base[i] = acc;
                        acc += V - __popcll(sm.tmask[i]);
                    }
                    sm.row_base[ns] = acc;
                }
                __syncthreads();
                const int R = sm.row_base[ns];
                for (int r = tid; r < R; r += NT) {
                    int i = 0;
                    while (sm.row_base[i + 1] <= r) ++i;
                    const int kth = r - sm.row_base[i];
                    const int t = select_bit(~sm.tmask[i] & full, kth);
                    const int64_t grow = a.rec_offsets[s0 + i] + kth;
                    const int mt = sm.msk[t];
                    const int kn = sm.known[t];
                    double pred[RS_NOPT];
                    long long key[RS_NOPT];
                    int validm = 0;
#pragma unroll
                    for (int j = 0; j < RS_NOPT; ++j) {
                        pred[j] = nan_d();
                        key[j] = 0;
                        const bool has = (mt >> j) & 1;
                        if (has && !(a.flags & RS_RANK_ALL)) continue;
                        const int f = i * RS_NOPT + j;
                        if (sm.status[f] != RS_FIT_OK) {
                            cnt[13] += 1;
                            continue;
                        }
                        const double* cf = sm.coef[f];
                        double yh = cf[0];
                        int aa = 1;
                        for (uint32_t x = sm.pmask[f]; x; x &= x - 1)
                            yh = fma(cf[aa++], sm.K[t * kKld + sm.pair_b[j][__ffs(x) - 1]], yh);
                        pred[j] = yh;
                        key[j] = okey(yh);
                        validm |= 1 << j;
                    }
                    const int scored = validm & kn;
                    cnt[1] += __popc(validm);
                    cnt[2] += __popc(scored);
                    // insertion sort of the valid candidates by key, descending; a later
                    // entry passes an earlier one only if strictly larger (ties: lower index)
                    int order[RS_NOPT];
                    int m = 0;
#pragma unroll
                    for (int j = 0; j < RS_NOPT; ++j)
                        if ((validm >> j) & 1) order[m++] = j;
                    for (int x = 1; x < m; ++x) {
                        const int cur = order[x];
                        int y = x - 1;
                        while (y >= 0 && key[order[y]] < key[cur]) {
                            order[y + 1] = order[y];
                            --y;
                        }
                        order[y + 1] = cur;
                    }
                    int c = 0;
                    uint32_t code = 0x0FFFFFF0u;
                    for (int x = 0; x < m && c < a.k; ++x) {
                        const int j = order[x];
                        if (key[j] >= ktau) {
                            code = (code & ~(0xFu << (4 + 4 * c))) | ((uint32_t)j << (4 + 4 * c));
                            if (a.rec_pred) a.rec_pred[grow * a.k + c] = pred[j];
                            ++c;
                        }
                    }
                    code = (code & ~0xFu) | (uint32_t)c;
                    a.rec_code[grow] = code;
                    if (a.rec_pred)
                        for (int x = c; x < a.k; ++x) a.rec_pred[grow * a.k + x] = nan_d();
                    if (a.pred_all)
#pragma unroll
                        for (int j = 0; j < RS_NOPT; ++j) a.pred_all[grow * RS_NOPT + j] = pred[j];
                    cnt[0] += 1;
                    cnt[4] += c;
                    int bp = -1, ba = -1;
#pragma unroll
                    for (int j = 0; j < RS_NOPT; ++j) {
                        if (!((scored >> j) & 1)) continue;
                        const long long ak = sm.act_key[t][j];
                        if ((key[j] > 0) == (ak > 0)) cnt[3] += 1;
                        if (bp < 0 || key[j] > key[bp]) bp = j;
                        if (ba < 0 || ak > sm.act_key[t][ba]) ba = j;
                    }
                    for (int x = 0; x < c; ++x) {
                        const int j = (code >> (4 + 4 * x)) & 0xF;
                        if ((scored >> j) & 1) {
                            cnt[5] += 1;
                            if (sm.act_key[t][j] > 0) cnt[6] += 1;
                        }
                    }
                    if (bp >= 0) {
                        cnt[7] += 1;
                        if (bp == ba) cnt[8] += 1;
                    }
                }
            }
            __syncthreads();
            s0 = seg_end;
        }
    }
    if (a.counters) {
#pragma unroll
        for (int c = 0; c < RS_NCOUNTERS; ++c) {
            const uint32_t v = __reduce_add_sync(0xffffffffu, cnt[c]);
            if (lane == 0 && v) atomicAdd(a.counters + c, (unsigned long long)v);
        }
    }
}

template <int WARPS, bool FIT>
cudaError_t launch_rank(const rs_fit_args& a, const int64_t* coef_off, const uint8_t* status_in,
                        cudaStream_t st) {
    using Sm = RankSmem<WARPS, FIT>;
    auto kern = rank_kernel<WARPS, FIT>;
    const size_t smem = sizeof(Sm);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t items = (a.S + kChunk - 1) / kChunk;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > items) grid = items;
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, WARPS * 32, smem, st>>>(a, coef_off, status_in);
    return cudaGetLastError();
}

// Workspace carve-up for the batched form.
struct FitWs {
    unsigned* hist;      // [kHist] fits per n
    unsigned* cursor;    // [kHist]
    unsigned long long* work;   // [4] work counters of the solve kernels
    uint8_t* pb;         // [P][6][32]
    uint8_t* pa;         // [P][6][32]
    double* ylab;        // [P][6][32]
    int* npair;          // [P][6]
    uint64_t* cand;      // [P][6]
    uint32_t* rowinfo;   // [P][64]
    uint64_t* pset;      // [P][6][kSetWords] the pairs' before and after slot sets, with their move masks
    uint8_t* psorted;    // [P] 1 when the program's masks ascend over its slots
    double* dlam;        // [P][64] K[t][t] + lambda
    unsigned long long* row_info;   // [Rcap] scoring summary | mask << 30
    int* split_prog;     // [S]
    uint32_t* fit_pm;    // [S*6]
    uint16_t* fit_key;   // [S*6] n * kCntBins + c
    uint4* recs;         // [S*6] fit records in bucket order
    int64_t* fit_off;    // [S*6]
    uint8_t* status;     // [S*6]
    double* coef;        // compact records
    double* predbuf;     // [6][Rcap]
    unsigned long long* tile_sum;   // [ceil(Rcap / 256)] recommendations per rank tile (packed output)
    unsigned long long* tile_off;   // [ceil(Rcap / 256)] their exclusive scan
    double* loo_tab;     // [P][6][kLooTab] M^-1, w_y, w_1, sums (RS_LOO_CLOSED; aliases coef)
    uint8_t* loo_ok;     // [P][6] 1 when that inverse exists
    uint32_t* loo_bad;   // [P][6] pairs whose label is not finite
    size_t bytes;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Row stride of the six prediction planes: even, so that every plane starts on a 16-byte
// boundary (the rank pass copies row ranges of the planes with TMA bulk copies).
int64_t plane_stride(int64_t Rcap) { return (Rcap + 1) & ~(int64_t)1; }

// histogram + bucket cursors (unsigned) and five 64-bit work counters, zeroed per call
constexpr size_t kCounterBytes = 2 * kHist * sizeof(unsigned) + 5 * sizeof(unsigned long long);

FitWs carve(void* base, int64_t P, int64_t S, int nmax, int64_t Rcap) {
    FitWs w{};
    char* c = (char*)base;
    size_t o = 0;
    auto take = [&](size_t b) { char* p = c ? c + o : nullptr; o += a256(b); return p; };
    const int64_t S6 = S * RS_NOPT;
    w.hist = (unsigned*)take(kCounterBytes);
    w.cursor = w.hist ? w.hist + kHist : nullptr;
    w.work = w.hist ? reinterpret_cast<unsigned long long*>(w.hist + 2 * kHist) : nullptr;
    w.pb = (uint8_t*)take(P * RS_NOPT * RS_MAXPAIRS);
    w.pa = (uint8_t*)take(P * RS_NOPT * RS_MAXPAIRS);
    w.ylab = (double*)take(P * RS_NOPT * RS_MAXPAIRS * sizeof(double));
    w.npair = (int*)take(P * RS_NOPT * sizeof(int));
    w.cand = (uint64_t*)take(P * RS_NOPT * sizeof(uint64_t));
    w.rowinfo = (uint32_t*)take(P * RS_MAXV * sizeof(uint32_t));
    w.pset = (uint64_t*)take(P * RS_NOPT * kSetWords * sizeof(uint64_t));
    w.psorted = (uint8_t*)take(P);
    w.dlam = (double*)take(P * RS_MAXV * sizeof(double));
    w.row_info = (unsigned long long*)take((size_t)Rcap * sizeof(unsigned long long));
    w.split_prog = (int*)take(S * sizeof(int));
    w.fit_pm = (uint32_t*)take(S6 * sizeof(uint32_t));
    w.fit_key = (uint16_t*)take(S6 * sizeof(uint16_t));
    w.recs = (uint4*)take(S6 * sizeof(uint4));
    w.fit_off = (int64_t*)take(S6 * sizeof(int64_t));
    w.status = (uint8_t*)take(S6);
    // compact records, or with RS_LOO_CLOSED (which keeps fits only in a caller's array) the
    // tables of the inverses: one region serves both
    const size_t coef_bytes = S6 * (size_t)(nmax + 1) * sizeof(double);
    const size_t loo_bytes = (size_t)P * RS_NOPT * kLooTab * sizeof(double);
    w.coef = (double*)take(coef_bytes > loo_bytes ? coef_bytes : loo_bytes);
    w.loo_tab = w.coef;
    w.predbuf = (double*)take((size_t)RS_NOPT * plane_stride(Rcap) * sizeof(double));
    const size_t ntiles = (size_t)((Rcap + kRankTile - 1) / kRankTile);
    w.tile_sum = (unsigned long long*)take(ntiles * sizeof(unsigned long long));
    w.tile_off = (unsigned long long*)take(ntiles * sizeof(unsigned long long));
    w.loo_ok = (uint8_t*)take(P * RS_NOPT);
    w.loo_bad = (uint32_t*)take(P * RS_NOPT * sizeof(uint32_t));
    w.bytes = o;
    return w;
}

template <int NLO, int NHI, int MINB>
cudaError_t launch_small(const SolveArgs& sa, int sms, int64_t S6, unsigned long long* work, cudaStream_t st) {
    auto kern = solve_small_kernel<NLO, NHI, MINB>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (S6 + 127) / 128;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, 128, 0, st>>>(sa, work);
    return cudaGetLastError();
}

// The one-fit-per-thread solver of kNReg < n <= nmax: as many warps per block as fit in
// 200 KB of shared memory (1..4), as many blocks as can be resident.
cudaError_t launch_mid(const SolveArgs& sa, int sms, int nmax, unsigned long long* work, cudaStream_t st) {
    const size_t per_warp = mid_warp_bytes(nmax);
    int warps = (int)((size_t)200 * 1024 / per_warp);
    if (warps > 4) warps = 4;
    if (warps < 1) warps = 1;
    const size_t smem = per_warp * warps;
    cudaError_t e = cudaFuncSetAttribute(solve_mid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_mid_kernel, warps * 32, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    solve_mid_kernel<<<(unsigned)grid, warps * 32, smem, st>>>(sa, nmax, work);
    return cudaGetLastError();
}

int nmax_of(int max_train) {
    int n = max_train / 2;   // pairs are disjoint in versions: at most half the train set
    if (n > RS_MAXPAIRS) n = RS_MAXPAIRS;
    if (n < 1) n = 1;
    return n;
}

}  // namespace

size_t rs_fit_workspace_bytes_impl(int64_t P, int64_t S, int max_train, int64_t Rcap) {
    return carve(nullptr, P, S, nmax_of(max_train), Rcap).bytes;
}

cudaError_t rs_launch_fit_predict(const rs_fit_args& a, cudaStream_t st) {
    if (a.S == 0) return cudaSuccess;
    if (a.form == RS_FORM_PLAIN) return launch_rank<8, true>(a, nullptr, nullptr, st);
    if (a.coef_in) return launch_rank<8, false>(a, nullptr, nullptr, st);
    // batched form: pairs -> plan -> bucket -> solve (+ predictions) -> rank pass
    if (!a.workspace) return cudaErrorInvalidValue;
    const int nmax = nmax_of(a.max_train);
    FitWs w = carve(a.workspace, a.P, a.S, nmax, a.rows_cap);
    if (w.bytes > a.workspace_bytes) return cudaErrorInvalidValue;
    const int64_t S6 = a.S * RS_NOPT;
    auto mark = [&](int i) { if (a.ev) cudaEventRecord(a.ev[i], st); };
    const bool plan = a.phase != 2, solve = a.phase != 1;
    cudaError_t e = cudaSuccess;
    const unsigned bucket_blocks = (unsigned)((S6 + kBucketThreads * kBucketPer - 1) / (kBucketThreads * kBucketPer));
    const bool user = a.coef_out != nullptr;
    uint8_t* status = a.status_out ? a.status_out : w.status;
    const bool rank = a.rec_code != nullptr;
    // compact records (and their offsets) only for fits without predictions or caller array
    const bool need_off = !user && !rank;
    if (plan) {
        e = cudaMemsetAsync(w.hist, 0, kCounterBytes, st);
        if (e != cudaSuccess) return e;
        mark(0);
        pairs_kernel<<<a.P, 64, 0, st>>>(a.P, a.row_offsets, a.masks, a.log_time, w.pb, w.pa, w.ylab,
                                         w.npair, w.cand, w.rowinfo, w.pset, w.psorted, a.dstatus);
        mark(1);
        plan_fits_kernel<<<(unsigned)((a.S + 255) / 256), 256, 0, st>>>(a.P, a.row_offsets, a.split_offsets, a.train_masks,
                                                    a.S, w.pb, w.pa, w.npair, w.fit_pm, w.fit_key, w.hist,
                                                    nmax, w.split_prog, a.rec_offsets,
                                                    a.rec_code ? a.rows_cap : 0,
                                                    a.rec_code ? w.row_info : nullptr,
                                                    a.masks, w.rowinfo, w.cand, (a.flags & RS_RANK_ALL) ? 1 : 0,
                                                    a.rec_code ? 1 : 0, w.pset, w.psorted, a.dstatus);
        mark(2);
        bucket_fits_kernel<<<bucket_blocks, kBucketThreads, 0, st>>>(S6, w.fit_key, w.hist, w.cursor, w.recs,
                                                      need_off ? w.fit_off : nullptr,
                                                      status, user ? a.coef_out : nullptr, a.counters,
                                                      w.fit_pm, w.split_prog, a.row_offsets);
        mark(3);
    }
    if (!solve) return cudaGetLastError();
    dlam_kernel<<<a.P, 64, 0, st>>>(a.row_offsets, a.K, a.lambda, w.dlam);
    if (!plan) mark(3);                        // the solvers start here, on this stream
    SolveArgs sa{a.P, a.split_offsets, w.split_prog, a.K, w.pb, w.ylab, w.fit_pm, w.fit_key, w.recs, w.hist,
                 w.fit_off, user ? a.coef_out : w.coef, user ? 1 : 0, status, a.lambda, w.dlam,
                 a.counters,
                 a.row_offsets, a.train_masks, a.rec_offsets, w.cand, rank ? w.predbuf : nullptr,
                 a.rows_cap, plane_stride(a.rows_cap), a.flags, a.dstatus, a.Z, a.x_offsets,
                 a.feat_width, a.max_feat, a.tune_order, rank ? w.row_info : nullptr};
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool refine = (a.flags & RS_REFINE_X) != 0;
    if (a.flags & RS_MODEL_IBK) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ibk_kernel, 128, 0);
        if (e != cudaSuccess) return e;
        int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
        const int64_t need = (S6 + 127) / 128;
        if (grid > need) grid = need;
        if (grid < 1) grid = 1;
        ibk_kernel<<<(unsigned)grid, 128, 0, st>>>(sa, nmax, w.work + 3);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        mark(4);
    } else if (a.flags & RS_LOO_CLOSED) {
        // one inverse per (program, optimization), then every fit in closed form
        loo_inv_kernel<<<(unsigned)(a.P * RS_NOPT), 32, 0, st>>>(a.row_offsets, a.K, w.pb, w.ylab, w.npair,
                                                                 w.dlam, w.loo_tab, w.loo_ok, w.loo_bad);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t grid = (S6 + kLooFitThreads - 1) / kLooFitThreads;
        loo_fit_kernel<<<(unsigned)grid, kLooFitThreads, 0, st>>>(sa, S6, w.npair, w.loo_tab, w.loo_ok, w.loo_bad);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        mark(4);
    } else if (!refine) {
        // Solvers over disjoint ranges of the bucket order.  The larger fits -- one thread per
        // fit from shared memory for kNReg < n <= kNMid (four warps per block fit), one warp per
        // fit above that (a thread's factor would no longer leave room for more than one warp
        // per SM) -- run on the side stream when there is one, beside the two register solvers
        // (n <= split, then split < n <= kNReg) on the call's stream; all take their work
        // dynamically, so the kernels sharing the SMs cost none of them a statically assigned
        // share.
        const bool mid = nmax > kNReg;
        const bool fork = mid && a.side && a.fork && a.join;
        cudaStream_t s2 = fork ? a.side : st;
        if (fork) {
            e = cudaEventRecord(a.fork, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(a.side, a.fork, 0);
        }
        if (e == cudaSuccess && mid) e = launch_mid(sa, sms, nmax < kNMid ? nmax : kNMid, w.work + 2, s2);
        if (e == cudaSuccess && nmax > kNMid) {
            // kWideGroups fits per warp, persistent blocks taking their fits dynamically
            e = cudaFuncSetAttribute(solve_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWideSmem);
            int per_sm = 0;
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solve_wide_kernel, kWideWarps * 32, kWideSmem);
            if (e == cudaSuccess) {
                int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
                const int64_t need = (S6 + kWideWarps * kWideGroups - 1) / (kWideWarps * kWideGroups);
                if (grid > need) grid = need;
                if (grid < 1) grid = 1;
                solve_wide_kernel<<<(unsigned)grid, kWideWarps * 32, kWideSmem, s2>>>(sa, w.work + 4);
                e = cudaGetLastError();
            }
        }
        if (e == cudaSuccess && fork) e = cudaEventRecord(a.join, a.side);
        if (e != cudaSuccess) return e;
        unsigned long long* w0 = w.work;
        unsigned long long* w1 = w.work + 1;
        switch (a.tune_split) {
            case 4: e = launch_small<1, 4, 4>(sa, sms, S6, w0, st);
                    if (e == cudaSuccess) e = launch_small<5, kNReg, 2>(sa, sms, S6, w1, st); break;
            case 5: e = launch_small<1, 5, 4>(sa, sms, S6, w0, st);
                    if (e == cudaSuccess) e = launch_small<6, kNReg, 2>(sa, sms, S6, w1, st); break;
            case 7: e = launch_small<1, 7, 3>(sa, sms, S6, w0, st);
                    if (e == cudaSuccess) e = launch_small<8, kNReg, 2>(sa, sms, S6, w1, st); break;
            case 8: e = launch_small<1, 8, 3>(sa, sms, S6, w0, st);
                    if (e == cudaSuccess) e = launch_small<9, kNReg, 2>(sa, sms, S6, w1, st); break;
            default: e = launch_small<1, 6, 4>(sa, sms, S6, w0, st);
                    if (e == cudaSuccess) e = launch_small<7, kNReg, 2>(sa, sms, S6, w1, st); break;
        }
        if (e != cudaSuccess) return e;
        mark(4);
        if (fork) {
            e = cudaStreamWaitEvent(st, a.join, 0);
            if (e != cudaSuccess) return e;
        }
    } else {
        mark(4);
        // refinement through Z: every fit by one warp (solve_large_kernel)
        const size_t lsmem = (size_t)kLargeWarps * 32 * 33 * sizeof(double) +
                             (size_t)kLargeWarps * (a.max_feat + 64 + 16) * sizeof(double);
        e = cudaFuncSetAttribute(solve_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem);
        if (e != cudaSuccess) return e;
        solve_large_kernel<<<(unsigned)(sms * 4), kLargeWarps * 32, lsmem, st>>>(sa);
    }
    mark(5);
    if (rank) {
        RankPassArgs ra{a.rec_offsets, a.S, w.predbuf, a.rows_cap, plane_stride(a.rows_cap), w.row_info,
                        a.dstatus, a.k, 0, a.flags, a.rec_code, a.rec_pred, a.pred_all, a.counters};
        ra.ktau = okey_host(a.log_tau);
        const bool packed = (a.flags & RS_PACK_PRED) != 0 && a.rec_pred != nullptr;
        const int64_t tiles_cap = (a.rows_cap + kRankTile - 1) / kRankTile;
        if (packed) {
            ra.pack_dst = w.predbuf;
            ra.tile_sum = w.tile_sum;
            e = cudaMemsetAsync(w.tile_sum, 0, (size_t)tiles_cap * sizeof(unsigned long long), st);
            if (e != cudaSuccess) return e;
        }
        auto rank_kern = packed ? rank_pass_kernel<true> : rank_pass_kernel<false>;
        e = cudaFuncSetAttribute(rank_kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRankSmem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rank_kern, kRankThreads, kRankSmem);
        if (e != cudaSuccess) return e;
        // persistent: tune_rank_waves (8, 16, 32) scales the resident blocks per SM by 1/4, 1/2, 1
        int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
        const int waves = a.tune_rank_waves > 0 ? a.tune_rank_waves : 32;
        blocks = blocks * waves / 32;
        const int64_t tiles = (a.rows_cap + kRankTile - 1) / kRankTile;
        if (blocks > tiles) blocks = tiles;
        if (blocks < 1) blocks = 1;
        rank_kern<<<(unsigned)blocks, kRankThreads, kRankSmem, st>>>(ra);
        if (packed && tiles_cap > 0) {
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            tile_scan_kernel<<<1, kScanThreads, 0, st>>>(w.tile_sum, w.tile_off, tiles_cap);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            pack_pred_kernel<<<(unsigned)tiles_cap, kRankTile, 0, st>>>(a.rec_offsets, a.S, a.rows_cap, a.rec_code,
                                                                        w.predbuf, plane_stride(a.rows_cap),
                                                                        w.tile_off, a.rec_pred);
        }
    }
    mark(6);
    return cudaGetLastError();
}
