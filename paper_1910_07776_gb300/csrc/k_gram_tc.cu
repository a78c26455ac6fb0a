// K2 (tensor-core form): per-program Gram K_p = Z_p Z_p^T from a BF16 hi/lo split of Z on the
// tcgen05 tensor cores, FP32 accumulation in tensor memory.
//
// z = hi + lo with hi = bf16(z) and lo = bf16(z - hi) carries about 16 significant bits; the
// Gram keeps three of the four products, K ~ hi hi^T + hi lo^T + lo hi^T (the dropped lo lo^T
// is ~2^-16 relative), which is ONE GEMM over a K dimension three times the feature width:
//      A_p = [hi | hi | lo],  B_p = [hi | lo | hi]   (rows = versions, zero-padded to 64),
//      K_p = A_p B_p^T.
// A prep kernel writes A and B for every program into a [P][64][3 F64] BF16 workspace (F64 =
// the widest feature count rounded up to 64); one batched launch (CTA z = program z, rank-3
// tensor maps) runs the GEMM; the epilogue converts to FP64 and writes a symmetric block (the
// entry (a, b), a <= b, is written to both places by one thread).
#include "tc_gemm.cuh"

namespace {

__global__ void __launch_bounds__(256)
split_kernel(int P, const int64_t* __restrict__ row_off, const int32_t* __restrict__ fw,
             const int64_t* __restrict__ xo, const double* __restrict__ Z, int Fp,
             __nv_bfloat16* A, __nv_bfloat16* B) {
    const int p = blockIdx.y;
    const int r = blockIdx.x;                       // version slot 0..63
    const int V = (int)(row_off[p + 1] - row_off[p]);
    const int F = fw[p];
    const int64_t base = ((int64_t)p * RS_MAXV + r) * 3 * Fp;
    for (int f = threadIdx.x; f < Fp; f += blockDim.x) {
        float zf = 0.f;
        if (r < V && V <= RS_MAXV && f < F) zf = (float)Z[xo[p] + (int64_t)r * F + f];
        const __nv_bfloat16 hi = __float2bfloat16(zf);
        const __nv_bfloat16 lo = __float2bfloat16(zf - __bfloat162float(hi));
        A[base + f] = hi;
        A[base + Fp + f] = hi;
        A[base + 2 * Fp + f] = lo;
        B[base + f] = hi;
        B[base + Fp + f] = lo;
        B[base + 2 * Fp + f] = hi;
    }
}

struct EpiGram {
    const int64_t* row_off;
    double* K;
    __device__ void operator()(int p, int row, int col0, const float (&v)[16]) const {
        const int V = (int)(row_off[p + 1] - row_off[p]);
        if (row >= V) return;
        double* Kp = K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int col = col0 + i;
            if (col < V && col >= row) {
                Kp[row * RS_GRAM_LD + col] = (double)v[i];
                Kp[col * RS_GRAM_LD + row] = (double)v[i];
            }
        }
    }
};

int padded_width(int max_feat) { return (max_feat + 63) / 64 * 64; }

}  // namespace

size_t rs_gram_tc_workspace_bytes(int64_t P, int max_feat) {
    return (size_t)2 * P * RS_MAXV * 3 * padded_width(max_feat) * sizeof(__nv_bfloat16) + 256;
}

cudaError_t rs_launch_gram_bf16x3_ws(const rs_batch* b, double* K, void* ws, size_t ws_bytes, int* dstatus,
                                     cudaStream_t st) {
    const int64_t P = b->n_programs;
    const int Fp = padded_width(b->max_feat);
    if (!ws || ws_bytes < rs_gram_tc_workspace_bytes(P, b->max_feat)) return cudaErrorInvalidValue;
    if (P > 65535) return cudaErrorInvalidValue;
    __nv_bfloat16* A = (__nv_bfloat16*)ws;
    __nv_bfloat16* B = A + (size_t)P * RS_MAXV * 3 * Fp;
    split_kernel<<<dim3(RS_MAXV, (unsigned)P), 256, 0, st>>>((int)P, b->row_offsets, b->feat_width,
                                                             b->x_offsets, (const double*)b->X, Fp, A, B);
    CUtensorMap ta, tb;
    cudaError_t e = rs_make_tmap_bf16_3d(&ta, A, P, RS_MAXV, 3 * Fp, 3 * Fp, tc::BM);
    if (e == cudaSuccess) e = rs_make_tmap_bf16_3d(&tb, B, P, RS_MAXV, 3 * Fp, 3 * Fp, RS_MAXV);
    if (e != cudaSuccess) return e;
    return tc::gemm_launch<64, 4, EpiGram, true>(ta, tb, RS_MAXV, RS_MAXV, 3 * Fp, (int)P,
                                                  EpiGram{b->row_offsets, K}, dstatus, st);
}
