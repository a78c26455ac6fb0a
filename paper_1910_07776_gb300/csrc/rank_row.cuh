// rank_row.cuh -- device pieces shared by the batched predict/rank path (k_fit.cu) and the
// transfer path (k_transfer.cu): order keys of doubles, FP64 reciprocals with few FP64
// instructions, the scoring summary of a version, and the ranking, threshold, top-k and
// scoring of one test row (Sec. 2 tier 3, Sec. 5, Sec. 6), plus the neighbour list of the
// instance-based learner.
#pragma once
#include <string.h>

#include "rs_internal.cuh"

namespace {

constexpr long long kNaNBits = 0x7ff8000000000000ll;

__device__ __forceinline__ double nan_d() { return __longlong_as_double(kNaNBits); }

// x > 0 and finite, decided on the bit pattern (no FP64 instruction).
__device__ __forceinline__ bool pos_finite(double x) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b < 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool finite_bits(double x) {
    return (__double_as_longlong(x) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}
// Order-preserving integer key of a non-NaN double: the bit pattern for a positive sign, minus
// the magnitude bits for a negative one (so -0.0 and +0.0 share key 0, and every key is above
// INT64_MIN).  For a negative sign b - INT64_MIN is the magnitude, so the key is INT64_MIN - b
// in wrapping arithmetic; no mask of the sign bit appears, which a compiler may turn into an
// FP64 absolute value (an instruction of the slow FP64 pipe).
__device__ __forceinline__ long long okey(double x) {
    const long long b = __double_as_longlong(x);
    return b < 0 ? (long long)(0x8000000000000000ull - (unsigned long long)b) : b;
}

// float <-> double for values inside the float normal range, by re-packing the IEEE-754
// fields with integer operations (the mantissa is truncated).  Used only to seed Newton
// iterations, so no FP64 instruction is spent on the conversion.
__device__ __forceinline__ float f32_of(double d) {
    const long long b = __double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    const unsigned m = (unsigned)((b >> 29) & 0x7fffff);
    return __uint_as_float(((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)e << 23) | m);
}
__device__ __forceinline__ double f64_of(float f) {
    const unsigned u = __float_as_uint(f);
    const long long e = (long long)((u >> 23) & 0xff) - 127 + 1023;
    return __longlong_as_double(((long long)(u & 0x80000000u) << 32) | (e << 52) |
                                ((long long)(u & 0x7fffff) << 29));
}

// 1/sqrt(d) for a positive finite d: FP32 seed, then two Newton steps of r <- r (3 - d r^2) / 2
// (Newton's method on f(r) = r^-2 - d).  The second step takes the residual 1/2 - (d/2) r^2
// from the exact square r^2 = s + s_lo (s_lo = fma(r, r, -s), Dekker's product), so the
// correction r e adds no more than the final rounding of r + r e.  Outside [1e-30, 1e30]:
// plain division.
__device__ __forceinline__ double rsqrt_newton(double d) {
    if (d < 1e-30 || d > 1e30) return 1.0 / sqrt(d);
    const double hd = 0.5 * d;
    double r = f64_of(rsqrtf(f32_of(d)));
    r = r * fma(-hd, r * r, 1.5);
    const double s = r * r;
    const double s_lo = fma(r, r, -s);
    const double e = fma(-hd, s_lo, fma(-hd, s, 0.5));
    return fma(r, e, r);
}

// Bit patterns of 2^-100 and 2^100 (positive doubles are ordered like their bit patterns).
constexpr long long kRcpLoBits = 0x39b0000000000000ll;
constexpr long long kRcpHiBits = 0x4630000000000000ll;

// 1/d for a positive finite d with three FP64 instructions.  r0 = the FP32 reciprocal of d
// (mantissa truncated to FP32) has relative error |t| < 2^-22 with t = 1 - d r0, and
// 1/d = r0 / (1 - t) = r0 (1 + t + t^2 + ...); keeping terms up to t^2 leaves |t|^3 < 2^-66,
// far below the final rounding:  t = fma(-d, r0, 1), u = fma(t, t, t), r = fma(r0, u, r0).
// The range test is an integer compare; outside [2^-100, 2^100]: plain division.
__device__ __forceinline__ double rcp_newton(double d) {
    const long long bits = __double_as_longlong(d);
    if (bits < kRcpLoBits || bits > kRcpHiBits) return 1.0 / d;
    const double r0 = f64_of(__frcp_rn(f32_of(d)));
    const double t = fma(-d, r0, 1.0);
    return fma(r0, fma(t, t, t), r0);
}

inline long long okey_host(double x) {
    long long b;
    memcpy(&b, &x, sizeof(b));
    const long long m = b & 0x7fffffffffffffffll;
    return b < 0 ? -m : m;
}

// Scoring summary of version t of a program (its masks msk, log times lt, and the slot of each
// mask, -1 if absent): bits 0-5 known (version t|j exists), bits 6-11 actual speedup > 1,
// bits 12-29 the six optimizations ordered by actual log speedup (descending, lower index
// first on ties, unknown last), 3 bits each.  t >= V gives the summary of an empty row.
__device__ __forceinline__ uint32_t row_summary(int t, int V, const uint8_t* msk, const double* lt,
                                                const int8_t* slot_of) {
    long long key[RS_NOPT];
    int kn = 0, apos = 0;
    for (int j = 0; j < RS_NOPT; ++j) {
        key[j] = (long long)0x8000000000000000ull;
        if (t < V && !((msk[t] >> j) & 1)) {
            const int w = slot_of[msk[t] | (1 << j)];
            if (w >= 0) {
                key[j] = okey(lt[t] - lt[w]);
                kn |= 1 << j;
                apos |= (key[j] > 0) << j;
            }
        }
    }
    uint32_t ord = 0;
    int used = 0;
    for (int x = 0; x < RS_NOPT; ++x) {
        int best = -1;
        for (int j = 0; j < RS_NOPT; ++j)
            if (!((used >> j) & 1) && (best < 0 || key[j] > key[best])) best = j;
        used |= 1 << best;
        ord |= (uint32_t)best << (3 * x);
    }
    return (uint32_t)kn | ((uint32_t)apos << 6) | (ord << 12);
}

constexpr int kIbkK = RS_IBK_NEIGHBORS;   // neighbours of the instance-based learner

struct RankPassArgs {
    const int64_t* rec_offsets;
    int64_t S;
    const double* predbuf;       // [6][PS]
    int64_t R;                   // rows of the buffer
    int64_t PS;                  // plane stride (even)
    const unsigned long long* row_info;  // [R] scoring summary | version mask << 30
    int* dstatus;
    int k;
    long long ktau;
    int flags;
    uint32_t* rec_code;
    double* rec_pred;
    double* pred_all;
    unsigned long long* counters;
    // packed predictions (RS_PACK_PRED): a row's chosen predictions go to its slots of the
    // prediction planes (pack_dst[pos * PS + row], already read by then) and each tile's
    // number of recommendations is added to tile_sum; a compaction pass writes rec_pred
    double* pack_dst;
    unsigned long long* tile_sum;
};

// Per-thread tallies of the scoring counters.
struct RankTally {
    uint32_t rows = 0, pred = 0, scored = 0, sign = 0, rec = 0, reck = 0, rech = 0, t1 = 0, t1h = 0, inv = 0;
};

// Ranking, threshold, top-k, outputs and scoring of one test row (Sec. 2 tier 3, Sec. 6):
// candidates (versions lacking j, or all with RS_RANK_ALL) whose fit succeeded are ranked by
// their predictions as order-preserving integer keys (ties: lower j first); those at or
// above log tau form the recommendation, the first k of them reported.  15 comparisons give,
// for each candidate j, the set of candidates that rank before it; its place is the
// popcount of that set restricted to the candidates at or above the threshold.
// info64: the row's scoring summary (row_summary) | version mask << 30 | mask of the
// optimizations whose fit has no training pair or failed << 36.  STAGE (k = STAGE_K): the
// reported values go to so[0 .. k-1] (the caller's shared-memory slots of the row) instead of
// rec_pred.
template <bool PACK = false, bool STAGE = false, int STAGE_K = 3>
__device__ __forceinline__ int rank_row(const RankPassArgs& a, int64_t row, unsigned long long info64,
                                        const double (&pred)[RS_NOPT], RankTally& c,
                                        double* so = nullptr) {
    const uint32_t info = (uint32_t)info64;
    const int mt = (int)(info64 >> 30) & 63;
    const int candm = (a.flags & RS_RANK_ALL) ? 63 : (~mt & 63);
    // a candidate counts when its fit had a training pair and did not fail (row record)
    const int okm = ~(int)(info64 >> 36) & 63;
    const int validm = candm & okm;
    long long key[RS_NOPT];
    int above = 0, spos = 0;
#pragma unroll
    for (int j = 0; j < RS_NOPT; ++j) {
        key[j] = okey(pred[j]);
        above |= (key[j] >= a.ktau) << j;
        spos |= (key[j] > 0) << j;
    }
    above &= validm;
    int bm[RS_NOPT];                           // bm[j]: candidates ranking before j
#pragma unroll
    for (int j = 0; j < RS_NOPT; ++j) bm[j] = 0;
#pragma unroll
    for (int i = 0; i < RS_NOPT; ++i)
#pragma unroll
        for (int j = i + 1; j < RS_NOPT; ++j) {
            if (key[i] >= key[j]) bm[j] |= 1 << i;
            else bm[i] |= 1 << j;
        }
    uint32_t code = 0x0FFFFFF0u;
    int rk = 0;
    int pos[RS_NOPT];
#pragma unroll
    for (int j = 0; j < RS_NOPT; ++j) {
        pos[j] = __popc(bm[j] & above);
        if (((above >> j) & 1) && pos[j] < a.k) {
            code = (code & ~(0xFu << (4 + 4 * pos[j]))) | ((uint32_t)j << (4 + 4 * pos[j]));
            rk |= 1 << j;
        }
    }
    const int nrec = __popc(rk);
    code = (code & ~0xFu) | (uint32_t)nrec;
    a.rec_code[row] = code;
    if constexpr (PACK) {                      // packed: park the list in the row's plane slots
#pragma unroll
        for (int j = 0; j < RS_NOPT; ++j)
            if ((rk >> j) & 1) a.pack_dst[pos[j] * a.PS + row] = pred[j];
    } else if constexpr (STAGE) {              // every slot, then each chosen candidate's
#pragma unroll
        for (int x = 0; x < STAGE_K; ++x) so[x] = nan_d();
#pragma unroll
        for (int j = 0; j < RS_NOPT; ++j)
            if ((rk >> j) & 1) so[pos[j]] = pred[j];
    } else if (a.rec_pred) {                   // each chosen candidate writes its own slot
        double* o = a.rec_pred + row * a.k;
#pragma unroll
        for (int j = 0; j < RS_NOPT; ++j)
            if ((rk >> j) & 1) o[pos[j]] = pred[j];
        for (int x = nrec; x < a.k; ++x) o[x] = nan_d();
    }
    if (a.pred_all)
#pragma unroll
        for (int j = 0; j < RS_NOPT; ++j)
            a.pred_all[row * RS_NOPT + j] = ((validm >> j) & 1) ? pred[j] : nan_d();
    const int known = info & 63, apos = (info >> 6) & 63;
    const int scored = validm & known;
    c.rows += 1;
    c.pred += __popc(validm);
    c.scored += __popc(scored);
    c.sign += __popc(scored & ~(spos ^ apos));
    c.rec += nrec;
    c.reck += __popc(rk & scored);
    c.rech += __popc(rk & scored & apos);
    c.inv += __popc(candm & ~okm);
    if (scored) {
        // ba: the scored optimization first in the actual order -- the order's first entry
        // when every known optimization is scored (unknown ones are ordered last)
        int ba = (info >> 12) & 7;
        if (scored != known) {
#pragma unroll
            for (int x = RS_NOPT - 1; x >= 0; --x) {
                const int j = (info >> (12 + 3 * x)) & 7;
                if ((scored >> j) & 1) ba = j;
            }
        }
        // a top-1 hit: no scored optimization is ranked before ba by the predictions
        int bmba = bm[0];
#pragma unroll
        for (int j = 1; j < RS_NOPT; ++j) bmba = ba == j ? bm[j] : bmba;
        c.t1 += 1;
        c.t1h += !(bmba & scored);
    }
    return nrec;
}

// Insertion of (d, q) into the list of the kIbkK nearest, ordered by (distance, index):
// distances are non-negative, so their bit patterns order like the values; a candidate
// replaces the last entry only when strictly nearer.
__device__ __forceinline__ void ibk_insert(unsigned long long (&kd)[kIbkK], int (&kq)[kIbkK],
                                           unsigned long long d, int q) {
    if (d >= kd[kIbkK - 1]) return;
#pragma unroll
    for (int i = kIbkK - 1; i > 0; --i) {
        const bool shift = kd[i - 1] > d;
        const bool here = !shift && kd[i] > d;
        kd[i] = shift ? kd[i - 1] : (here ? d : kd[i]);
        kq[i] = shift ? kq[i - 1] : (here ? q : kq[i]);
    }
    if (kd[0] > d) {
        kd[0] = d;
        kq[0] = q;
    }
}

}  // namespace
