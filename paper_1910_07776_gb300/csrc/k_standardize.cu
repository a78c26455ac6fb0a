// K1: feature vectors (Sec. 2: counters normalised by the cycle count), followed by the
// library's log / per-program z-score reading.  One read of X, one write of Z.
//
// The logarithm runs once per element on this part's narrow FP64 pipe, so it is written
// here to need few FP64 instructions (log_pos below, 9 of them); X is read once, spread
// over sixteen row groups per feature, in blocks small enough (16 features) that programs
// of different sizes spread evenly over the SMs.
#include "rs_internal.cuh"
#include "rs_log_table.h"

namespace {

constexpr long long kClampBits = 0x39b4484bfeebc2a0ll;   // bit pattern of 1e-30
constexpr long long kInfBits = 0x7ff0000000000000ll;

// log q for a positive, normal, finite q, table-driven (after P. T. P. Tang, "Table-driven
// implementation of the logarithm function in IEEE floating-point arithmetic", ACM TOMS
// 16(4), 1990): q = 2^e m with m in [1, 2); F = the centre of m's interval of width 1/256
// (index i = the top eight fraction bits of m); r = m (1/F) - 1 in one FMA, |r| <= 2^-9;
//     log q = e ln2 + (log F + log1p(r)),
// log1p(r) by its Taylor series up to r^5 (the first term left out, r^6 / 6, is below
// 2^-56), e ln2 as one FMA with ln 2 rounded to FP64.  9 FP64 instructions.  Against an
// extended-precision log over 3e7 arguments (1e-29 .. 1e31, exponents -1000 .. 1000, and
// q within 0.5 % of 1) the error is at most 2.4 units of 2^-53 max(1, |log q|), rms 0.52 --
// the same as Tang's exact reduction m - F and split ln 2 (2.2, rms 0.51), which took three
// more FP64 instructions.
__device__ __forceinline__ double log_pos(double q, const double* tlog, const double* tinv) {
    const long long b = __double_as_longlong(q);
    const int i = (int)((b >> 44) & 0xff);
    const double m = __longlong_as_double((b & 0x000fffffffffffffll) | 0x3ff0000000000000ll);
    const double r = fma(m, tinv[i], -1.0);
    double p = fma(r, 0.2, -0.25);
    p = fma(p, r, 1.0 / 3.0);
    p = fma(p, r, -0.5);
    const double l1p = fma(r * r, p, r);
    // e as a double without a conversion instruction: 2^52 + 2048 + e, minus 2^52 + 2048
    const long long eb = (b >> 52) - 1023 + 2048;
    const double ed = __longlong_as_double(0x4330000000000000ll | eb) - 4503599627372544.0;
    return fma(ed, kLn2, tlog[i] + l1p);
}

// log(max(q, 1e-30)) with the branches of the plain definition: q above the clamp and finite
// -> log_pos (subnormal q never reach it); +inf -> +inf; q <= 1e-30 or NaN -> log(1e-30).
__device__ __forceinline__ double log_clamped(double q, const double* tlog, const double* tinv) {
    const long long b = __double_as_longlong(q);
    if (b > kClampBits && b < kInfBits) return log_pos(q, tlog, tinv);
    return b == kInfBits ? q : kLogClamp;
}

// An input element as a double: FP32 values are re-packed with integer operations (exact for
// normal numbers); zeros, subnormals, infinities and NaNs take the conversion instruction.
__device__ __forceinline__ double as_double(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned ex = (u >> 23) & 0xff;
    if (ex == 0 || ex == 0xff) return (double)x;
    return __longlong_as_double(((long long)(u & 0x80000000u) << 32) |
                                ((long long)(ex - 127 + 1023) << 52) | ((long long)(u & 0x7fffff) << 29));
}
__device__ __forceinline__ double as_double(double x) { return x; }

constexpr int kFeat = 16;                    // features per block
constexpr int kGroups = 16;                  // row groups per block
constexpr int kThreads = kFeat * kGroups;

// Block = (program, 16-feature slice); thread (g, f) takes rows g, g + 16, ... of feature f.
// A warp reads 16 consecutive features of two rows (64-byte segments).  The log values stay in
// shared memory; per-feature sums are combined from the 16 row groups in a fixed order.
template <typename T>
__global__ void __launch_bounds__(kThreads)
standardize_kernel(int P, const int64_t* __restrict__ row_off, const int32_t* __restrict__ fw,
                   const int64_t* __restrict__ xo, const int64_t* __restrict__ fo,
                   const T* __restrict__ X, const double* __restrict__ cycles,
                   double* __restrict__ Z, double* __restrict__ mu, double* __restrict__ sigma,
                   int* dstatus) {
    __shared__ double lv[RS_MAXV][kFeat];
    __shared__ double part[kGroups][kFeat];
    __shared__ double stat[2][kFeat];
    __shared__ double inv_c[RS_MAXV];
    __shared__ double tlog[256], tinv[256];
    const int p = blockIdx.x;
    const int64_t r0 = row_off[p];
    const int V = (int)(row_off[p + 1] - r0);
    const int F = fw[p];
    const int fl = threadIdx.x % kFeat, g = threadIdx.x / kFeat;
    const int f = blockIdx.y * kFeat + fl;
    if (blockIdx.y * kFeat >= F) return;
    if (V < 1 || V > RS_MAXV) {
        if (threadIdx.x == 0 && blockIdx.y == 0) rs_dev_flag(dstatus, RS_EDATA, p);
        return;
    }
    const int64_t base = xo[p];
    const bool active = f < F;
    // one reciprocal per version instead of a division per element (FP64 divisions are
    // expensive on this part's narrow FP64 pipe)
    if (cycles && threadIdx.x < V) inv_c[threadIdx.x] = 1.0 / cycles[r0 + threadIdx.x];
    for (int t = threadIdx.x; t < 256; t += kThreads) {
        tlog[t] = kLogTabF[t];
        tinv[t] = kLogTabInv[t];
    }
    __syncthreads();
    double s = 0.0;
    if (active)
        for (int r = g; r < V; r += kGroups) {
            double x = as_double(X[base + (int64_t)r * F + f]);
            if (cycles) x = x * inv_c[r];
            const double l = log_clamped(x, tlog, tinv);
            lv[r][fl] = l;
            s += l;
        }
    part[g][fl] = s;
    __syncthreads();
    if (g == 0) {
        double t = 0.0;
        for (int q = 0; q < kGroups; ++q) t += part[q][fl];
        stat[0][fl] = t / V;
    }
    __syncthreads();
    const double m = stat[0][fl];
    double q2 = 0.0;
    if (active)
        for (int r = g; r < V; r += kGroups) {
            const double d = lv[r][fl] - m;
            lv[r][fl] = d;                     // kept for the output
            q2 += d * d;
        }
    part[g][fl] = q2;
    __syncthreads();
    if (g == 0) {
        double t = 0.0;
        for (int q = 0; q < kGroups; ++q) t += part[q][fl];
        stat[1][fl] = sqrt(t / V);
    }
    __syncthreads();
    if (!active) return;
    const double sd = stat[1][fl];
    const bool ok = sd > 1e-12;
    const double rs = ok ? 1.0 / sd : 0.0;
    for (int r = g; r < V; r += kGroups)
        Z[base + (int64_t)r * F + f] = ok ? lv[r][fl] * rs : 0.0;
    if (g == 0) {
        if (mu) mu[fo[p] + f] = m;
        if (sigma) sigma[fo[p] + f] = sd;
    }
}

// Standardization of the training side of a transfer (Table 2): problem q trains on the runs
// group_off[q] .. group_off[q+1]-1 (each laid out like one program: at most 64 versions, all
// with the width F of the problem's test program), standardized together -- mu, sigma over
// the vectors of all of them -- into Z in X's layout; mu, sigma at q * stat_stride + f.
// Block = (problem, 16-feature slice), as standardize_kernel with up to kGroupRows rows.
constexpr int kGroupRows = RS_MAXV * RS_MAXRUNS;

template <typename T>
__global__ void __launch_bounds__(kThreads)
group_standardize_kernel(const int64_t* __restrict__ group_off, int max_runs, int64_t n_runs,
                         const int64_t* __restrict__ row_off,
                         const int32_t* __restrict__ fw, const int64_t* __restrict__ xo,
                         const T* __restrict__ X, const double* __restrict__ cycles,
                         const int32_t* __restrict__ fw_test, int stat_stride, double* __restrict__ Z,
                         double* __restrict__ mu, double* __restrict__ sigma, int* dstatus) {
    __shared__ double lv[kGroupRows][kFeat];
    __shared__ double part[kGroups][kFeat];
    __shared__ double stat[2][kFeat];
    __shared__ double inv_c[kGroupRows];
    __shared__ int64_t rowx[kGroupRows];
    __shared__ double tlog[256], tinv[256];
    const int q = blockIdx.x;
    int start[RS_MAXRUNS + 1], F = 0;
    const int N = rs_group_layout(q, group_off, max_runs, n_runs, row_off, fw, fw_test, stat_stride, start, F);
    if (N < 0) {
        if (threadIdx.x == 0 && blockIdx.y == 0) rs_dev_flag(dstatus, RS_EDATA, q);
        return;
    }
    if (blockIdx.y * kFeat >= F) return;
    const int fl = threadIdx.x % kFeat, g = threadIdx.x / kFeat;
    const int f = blockIdx.y * kFeat + fl;
    const bool active = f < F;
    const int64_t g0 = group_off[q];
    for (int u = threadIdx.x; u < N; u += kThreads) {
        int r = 0;
        while (u >= start[r + 1]) ++r;
        const int v = u - start[r];
        rowx[u] = xo[g0 + r] + (int64_t)v * F;
        if (cycles) inv_c[u] = 1.0 / cycles[row_off[g0 + r] + v];
    }
    for (int t = threadIdx.x; t < 256; t += kThreads) {
        tlog[t] = kLogTabF[t];
        tinv[t] = kLogTabInv[t];
    }
    __syncthreads();
    double s = 0.0;
    if (active)
        for (int u = g; u < N; u += kGroups) {
            double x = as_double(X[rowx[u] + f]);
            if (cycles) x = x * inv_c[u];
            const double l = log_clamped(x, tlog, tinv);
            lv[u][fl] = l;
            s += l;
        }
    part[g][fl] = s;
    __syncthreads();
    if (g == 0) {
        double t = 0.0;
        for (int i = 0; i < kGroups; ++i) t += part[i][fl];
        stat[0][fl] = t / N;
    }
    __syncthreads();
    const double m = stat[0][fl];
    double q2 = 0.0;
    if (active)
        for (int u = g; u < N; u += kGroups) {
            const double d = lv[u][fl] - m;
            lv[u][fl] = d;                     // kept for the output
            q2 += d * d;
        }
    part[g][fl] = q2;
    __syncthreads();
    if (g == 0) {
        double t = 0.0;
        for (int i = 0; i < kGroups; ++i) t += part[i][fl];
        stat[1][fl] = sqrt(t / N);
    }
    __syncthreads();
    if (!active) return;
    const double sd = stat[1][fl];
    const bool ok = sd > 1e-12;
    const double rs = ok ? 1.0 / sd : 0.0;
    for (int u = g; u < N; u += kGroups) Z[rowx[u] + f] = ok ? lv[u][fl] * rs : 0.0;
    if (g == 0) {
        mu[(int64_t)q * stat_stride + f] = m;
        sigma[(int64_t)q * stat_stride + f] = sd;
    }
}

// The test side: program q standardized with its training group's statistics (at
// q * stat_stride + f): z = (log max(x / c, 1e-30) - mu) / sigma, or 0 where sigma <= 1e-12.
template <typename T>
__global__ void __launch_bounds__(kThreads)
standardize_apply_kernel(const int64_t* __restrict__ row_off, const int32_t* __restrict__ fw,
                         const int64_t* __restrict__ xo, const T* __restrict__ X,
                         const double* __restrict__ cycles, const double* __restrict__ mu,
                         const double* __restrict__ sigma, int stat_stride, double* __restrict__ Z) {
    __shared__ double inv_c[RS_MAXV];
    __shared__ double tlog[256], tinv[256];
    const int p = blockIdx.x;
    const int64_t r0 = row_off[p];
    const int V = (int)(row_off[p + 1] - r0);
    const int F = fw[p];
    const int fl = threadIdx.x % kFeat, g = threadIdx.x / kFeat;
    const int f = blockIdx.y * kFeat + fl;
    // a bad program was reported by group_standardize_kernel
    if (blockIdx.y * kFeat >= F || V < 1 || V > RS_MAXV || F > stat_stride) return;
    if (cycles && threadIdx.x < V) inv_c[threadIdx.x] = 1.0 / cycles[r0 + threadIdx.x];
    for (int t = threadIdx.x; t < 256; t += kThreads) {
        tlog[t] = kLogTabF[t];
        tinv[t] = kLogTabInv[t];
    }
    __syncthreads();
    if (f >= F) return;
    const double m = mu[(int64_t)p * stat_stride + f], sd = sigma[(int64_t)p * stat_stride + f];
    const bool ok = sd > 1e-12;
    const double rs = ok ? 1.0 / sd : 0.0;
    const int64_t base = xo[p];
    for (int r = g; r < V; r += kGroups) {
        double x = as_double(X[base + (int64_t)r * F + f]);
        if (cycles) x = x * inv_c[r];
        const double l = log_clamped(x, tlog, tinv);
        Z[base + (int64_t)r * F + f] = ok ? (l - m) * rs : 0.0;
    }
}

}  // namespace

cudaError_t rs_launch_transfer_standardize(const rs_batch* train, const rs_batch* test, const int64_t* group_off,
                                           int max_runs, int stat_stride, double* ZA, double* ZB, double* mu,
                                           double* sigma, int* dstatus, cudaStream_t st) {
    const int Q = test->n_programs;
    dim3 ga((unsigned)Q, (unsigned)((stat_stride + kFeat - 1) / kFeat));
    if (train->dtype == RS_F32)
        group_standardize_kernel<float><<<ga, kThreads, 0, st>>>(
            group_off, max_runs, train->n_programs, train->row_offsets, train->feat_width, train->x_offsets,
            (const float*)train->X,
            train->cycles, test->feat_width, stat_stride, ZA, mu, sigma, dstatus);
    else
        group_standardize_kernel<double><<<ga, kThreads, 0, st>>>(
            group_off, max_runs, train->n_programs, train->row_offsets, train->feat_width, train->x_offsets,
            (const double*)train->X,
            train->cycles, test->feat_width, stat_stride, ZA, mu, sigma, dstatus);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 gb((unsigned)Q, (unsigned)((test->max_feat + kFeat - 1) / kFeat));
    if (test->dtype == RS_F32)
        standardize_apply_kernel<float><<<gb, kThreads, 0, st>>>(test->row_offsets, test->feat_width, test->x_offsets,
                                                                 (const float*)test->X, test->cycles, mu, sigma,
                                                                 stat_stride, ZB);
    else
        standardize_apply_kernel<double><<<gb, kThreads, 0, st>>>(test->row_offsets, test->feat_width,
                                                                  test->x_offsets, (const double*)test->X,
                                                                  test->cycles, mu, sigma, stat_stride, ZB);
    return cudaGetLastError();
}

cudaError_t rs_launch_standardize(const rs_batch* b, double* Z, double* mu, double* sigma,
                                  int* dstatus, cudaStream_t st) {
    dim3 grid((unsigned)b->n_programs, (unsigned)((b->max_feat + kFeat - 1) / kFeat));
    if (b->dtype == RS_F32)
        standardize_kernel<float><<<grid, kThreads, 0, st>>>(
            b->n_programs, b->row_offsets, b->feat_width, b->x_offsets, b->feat_offsets,
            (const float*)b->X, b->cycles, Z, mu, sigma, dstatus);
    else
        standardize_kernel<double><<<grid, kThreads, 0, st>>>(
            b->n_programs, b->row_offsets, b->feat_width, b->x_offsets, b->feat_offsets,
            (const double*)b->X, b->cycles, Z, mu, sigma, dstatus);
    return cudaGetLastError();
}
