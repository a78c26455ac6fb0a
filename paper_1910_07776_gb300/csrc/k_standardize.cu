// K1: feature vectors (Sec. 2: counters normalised by the cycle count), followed by the
// library's log / per-program z-score reading.  HBM-bound: one read of X, one write of Z.
//
// Grid: (program, feature chunk).  Each thread owns one feature column of one program;
// a warp reads 32 consecutive features of a row (coalesced).  The V <= 64 log values of a
// column stay in shared memory between the three passes (sum, squared deviations, z), so
// X is read once and the FP64 log -- expensive on this part's FP64 pipe -- runs once per
// element.
#include "rs_internal.cuh"

namespace {

constexpr int kThreads = 64;   // 64 rows x 64 columns of doubles = 32 KiB of shared memory

template <typename T>
__global__ void __launch_bounds__(kThreads)
standardize_kernel(int P, const int64_t* __restrict__ row_off, const int32_t* __restrict__ fw,
                   const int64_t* __restrict__ xo, const int64_t* __restrict__ fo,
                   const T* __restrict__ X, const double* __restrict__ cycles,
                   double* __restrict__ Z, double* __restrict__ mu, double* __restrict__ sigma,
                   int* dstatus) {
    __shared__ double lv[RS_MAXV][kThreads];
    const int p = blockIdx.x;
    const int64_t r0 = row_off[p];
    const int V = (int)(row_off[p + 1] - r0);
    const int F = fw[p];
    const int f = blockIdx.y * kThreads + threadIdx.x;
    if (blockIdx.y * kThreads >= F) return;
    if (V < 1 || V > RS_MAXV) {
        if (threadIdx.x == 0 && blockIdx.y == 0) rs_dev_flag(dstatus, RS_EDATA, p);
        return;
    }
    const int64_t base = xo[p];
    const bool active = f < F;
    double s = 0.0;
    if (active) {
        for (int r = 0; r < V; ++r) {
            double x = (double)X[base + (int64_t)r * F + f];
            if (cycles) x = x / cycles[r0 + r];
            double l = log(x > 1e-30 ? x : 1e-30);
            lv[r][threadIdx.x] = l;
            s += l;
        }
    }
    const double m = s / V;
    double q = 0.0;
    if (active)
        for (int r = 0; r < V; ++r) {
            double d = lv[r][threadIdx.x] - m;
            q += d * d;
        }
    const double sd = sqrt(q / V);
    if (!active) return;
    const bool ok = sd > 1e-12;
    const double rs = ok ? 1.0 / sd : 0.0;
    for (int r = 0; r < V; ++r)
        Z[base + (int64_t)r * F + f] = ok ? (lv[r][threadIdx.x] - m) * rs : 0.0;
    if (mu) mu[fo[p] + f] = m;
    if (sigma) sigma[fo[p] + f] = sd;
}

}  // namespace

cudaError_t rs_launch_standardize(const rs_batch* b, double* Z, double* mu, double* sigma,
                                  int* dstatus, cudaStream_t st) {
    dim3 grid((unsigned)b->n_programs, (unsigned)((b->max_feat + kThreads - 1) / kThreads));
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
