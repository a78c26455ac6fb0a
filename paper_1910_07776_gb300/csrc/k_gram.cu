// K2 (FP64 form): per-program Gram block K_p = Z_p Z_p^T of the standardized feature
// vectors.  It is the only contraction of the method: every ridge fit of every split of
// program p reads its kernel entries K_p[v_a][v_b] from this block (dual form of the
// regression family of Sec. 3.4), so it is formed once per program, not once per fit.
//
// Grid: (program, upper-triangular 16x16 output tile); 10 tiles cover 64x64.  Each CTA
// streams both row panels through shared memory in 32-feature slices; each thread owns
// one output entry.  Off-diagonal tiles also write the mirrored entry.
#include "rs_internal.cuh"

namespace {

constexpr int kTile = 16;
constexpr int kSlice = 32;

__constant__ int2 kTilePairs[10] = {{0, 0}, {0, 1}, {0, 2}, {0, 3}, {1, 1},
                                    {1, 2}, {1, 3}, {2, 2}, {2, 3}, {3, 3}};

__global__ void __launch_bounds__(kTile * kTile)
gram_f64_kernel(int P, const int64_t* __restrict__ row_off, const int32_t* __restrict__ fw,
                const int64_t* __restrict__ xo, const double* __restrict__ Z,
                double* __restrict__ K, int* dstatus) {
    __shared__ double A[kTile][kSlice + 1];
    __shared__ double B[kTile][kSlice + 1];
    const int p = blockIdx.x;
    const int V = (int)(row_off[p + 1] - row_off[p]);
    if (V < 1 || V > RS_MAXV) {
        if (threadIdx.x == 0 && threadIdx.y == 0 && blockIdx.y == 0) rs_dev_flag(dstatus, RS_EDATA, p);
        return;
    }
    const int2 tp = kTilePairs[blockIdx.y];
    const int a0 = tp.x * kTile, b0 = tp.y * kTile;
    if (a0 >= V || b0 >= V) return;
    const int F = fw[p];
    const double* Zp = Z + xo[p];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTile + tx;
    double acc = 0.0;
    for (int f0 = 0; f0 < F; f0 += kSlice) {
        // 256 threads load 2 x 16 x 32 values: thread -> (row = tid / 32 [+8], col = tid % 32)
        for (int e = tid; e < kTile * kSlice; e += kTile * kTile) {
            const int r = e / kSlice, c = e % kSlice;
            const int f = f0 + c;
            const int ra = a0 + r, rb = b0 + r;
            A[r][c] = (ra < V && f < F) ? Zp[(int64_t)ra * F + f] : 0.0;
            B[r][c] = (rb < V && f < F) ? Zp[(int64_t)rb * F + f] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < kSlice; ++c) acc = fma(A[ty][c], B[tx][c], acc);
        __syncthreads();
    }
    const int a = a0 + ty, b = b0 + tx;
    if (a < V && b < V) {
        double* Kp = K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
        Kp[a * RS_GRAM_LD + b] = acc;
        if (a0 != b0) Kp[b * RS_GRAM_LD + a] = acc;
    }
}

}  // namespace

cudaError_t rs_launch_gram_f64(const rs_batch* b, double* K, int* dstatus, cudaStream_t st) {
    dim3 grid((unsigned)b->n_programs, 10);
    dim3 block(kTile, kTile);
    gram_f64_kernel<<<grid, block, 0, st>>>(b->n_programs, b->row_offsets, b->feat_width,
                                            b->x_offsets, (const double*)b->X, K, dstatus);
    return cudaGetLastError();
}
