// K1: feature vectors (Sec. 2: counters normalised by the cycle count), followed by the
// library's log / per-program z-score reading.  HBM-bound: one read of X, one write of Z.
//
// X is read once and the FP64 log -- expensive on this part's narrow FP64 pipe -- runs once
// per element, spread over eight row groups per feature so that every SM has FP64 work.
#include "rs_internal.cuh"

namespace {

constexpr int kFeat = 32;                    // features per block (one warp-wide row slice)
constexpr int kGroups = 8;                   // row groups per block
constexpr int kThreads = kFeat * kGroups;

// Block = (program, 32-feature slice); thread (g, f) takes rows g, g + 8, ... of feature f.
// A warp reads 32 consecutive features of one row (coalesced).  The log values stay in
// shared memory; per-feature sums are combined from the 8 row groups in a fixed order.
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
    __syncthreads();
    double s = 0.0;
    if (active)
        for (int r = g; r < V; r += kGroups) {
            double x = (double)X[base + (int64_t)r * F + f];
            if (cycles) x = x * inv_c[r];
            const double l = log(x > 1e-30 ? x : 1e-30);
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
        Z[base + (int64_t)r * F + f] = ok ? (lv[r][fl] - m) * rs : 0.0;
    if (g == 0) {
        if (mu) mu[fo[p] + f] = m;
        if (sigma) sigma[fo[p] + f] = sd;
    }
}

}  // namespace

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
