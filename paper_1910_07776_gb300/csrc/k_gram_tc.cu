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
// entry (a, b), a <= b, is written to both places by one thread).  Two tile choices, picked
// per padded feature width by the autotuner: the output tile's width (32 or 64 columns of the
// 64 x 64 block), and the K split (the whole K = 3 F64 in one CTA, or the three products on
// three CTAs with their FP32 results summed in FP64 in a fixed order).
#include "tc_gemm.cuh"

namespace {

// ksplit = 1: A_p = [hi | hi | lo], B_p = [hi | lo | hi] (one product, K = 3 Fp).
// ksplit = 3: the three products hi hi^T, hi lo^T, lo hi^T as three batches of K = Fp each
// (batch 3 p + r), whose FP32 results are summed in FP64 afterwards in a fixed order.
__global__ void __launch_bounds__(256)
split_kernel(int P, const int64_t* __restrict__ row_off, const int32_t* __restrict__ fw,
             const int64_t* __restrict__ xo, const double* __restrict__ Z, int Fp, int ksplit,
             __nv_bfloat16* A, __nv_bfloat16* B) {
    const int p = blockIdx.y;
    const int r = blockIdx.x;                       // version slot 0..63
    const int V = (int)(row_off[p + 1] - row_off[p]);
    const int F = fw[p];
    const int kw = 3 * Fp / ksplit;                 // K of one batch
    auto at = [&](int seg) {                        // element offset of segment seg of row r
        const int z = p * ksplit + seg * ksplit / 3;
        return ((int64_t)z * RS_MAXV + r) * kw + (int64_t)(seg % (3 / ksplit)) * Fp;
    };
    const int64_t s0 = at(0), s1 = at(1), s2 = at(2);
    for (int f = threadIdx.x; f < Fp; f += blockDim.x) {
        float zf = 0.f;
        if (r < V && V <= RS_MAXV && f < F) zf = (float)Z[xo[p] + (int64_t)r * F + f];
        const __nv_bfloat16 hi = __float2bfloat16(zf);
        const __nv_bfloat16 lo = __float2bfloat16(zf - __bfloat162float(hi));
        A[s0 + f] = hi;
        A[s1 + f] = hi;
        A[s2 + f] = lo;
        B[s0 + f] = hi;
        B[s1 + f] = lo;
        B[s2 + f] = hi;
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

// ksplit = 3: the FP32 result of batch z, rows and columns < 64.
struct EpiGramPart {
    float* part;
    __device__ void operator()(int z, int row, int col0, const float (&v)[16]) const {
        float* o = part + ((int64_t)z * RS_MAXV + row) * RS_MAXV + col0;
#pragma unroll
        for (int i = 0; i < 16; ++i) o[i] = v[i];
    }
};

// K_p[a][b] = part[3p][a][b] + part[3p+1][a][b] + part[3p+2][a][b], summed in FP64 in that
// order, written to both triangles from the upper one.
__global__ void __launch_bounds__(256)
gram_reduce_kernel(const int64_t* __restrict__ row_off, const float* __restrict__ part, double* K) {
    const int p = blockIdx.x;
    const int V = (int)(row_off[p + 1] - row_off[p]);
    const float* q = part + (int64_t)p * 3 * RS_MAXV * RS_MAXV;
    double* Kp = K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
    for (int e = threadIdx.x; e < RS_MAXV * RS_MAXV; e += blockDim.x) {
        const int a = e / RS_MAXV, b = e % RS_MAXV;
        if (a >= V || b >= V || b < a) continue;
        const double v = ((double)q[e] + (double)q[RS_MAXV * RS_MAXV + e]) + (double)q[2 * RS_MAXV * RS_MAXV + e];
        Kp[a * RS_GRAM_LD + b] = v;
        Kp[b * RS_GRAM_LD + a] = v;
    }
}

int padded_width(int max_feat) { return (max_feat + 63) / 64 * 64; }

template <int BN>
cudaError_t gram_gemm(const CUtensorMap& ta, const CUtensorMap& tb, int kw, int batch, int ksplit,
                      const rs_batch* b, double* K, float* part, int* dstatus, cudaStream_t st) {
    if (ksplit == 1)
        return tc::gemm_launch<BN, 4, EpiGram, true>(ta, tb, RS_MAXV, RS_MAXV, kw, batch, EpiGram{b->row_offsets, K},
                                                     dstatus, st);
    cudaError_t e = tc::gemm_launch<BN, 4, EpiGramPart, true>(ta, tb, RS_MAXV, RS_MAXV, kw, batch,
                                                              EpiGramPart{part}, dstatus, st);
    if (e == cudaSuccess) {
        gram_reduce_kernel<<<(unsigned)b->n_programs, 256, 0, st>>>(b->row_offsets, part, K);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

size_t rs_gram_tc_workspace_bytes(int64_t P, int max_feat) {
    return (size_t)2 * P * RS_MAXV * 3 * padded_width(max_feat) * sizeof(__nv_bfloat16) +
           (size_t)3 * P * RS_MAXV * RS_MAXV * sizeof(float) + 512;
}

cudaError_t rs_launch_gram_bf16x3_ws(const rs_batch* b, double* K, void* ws, size_t ws_bytes, int* dstatus,
                                     cudaStream_t st, int tile_n, int ksplit) {
    const int64_t P = b->n_programs;
    const int Fp = padded_width(b->max_feat);
    if (!ws || ws_bytes < rs_gram_tc_workspace_bytes(P, b->max_feat)) return cudaErrorInvalidValue;
    if (P > 65535 || (ksplit != 1 && ksplit != 3) || (tile_n != 32 && tile_n != 64)) return cudaErrorInvalidValue;
    const size_t half = (size_t)P * RS_MAXV * 3 * Fp;
    __nv_bfloat16* A = (__nv_bfloat16*)ws;
    __nv_bfloat16* B = A + half;
    float* part = (float*)(((uintptr_t)(B + half) + 255) & ~(uintptr_t)255);
    split_kernel<<<dim3(RS_MAXV, (unsigned)P), 256, 0, st>>>((int)P, b->row_offsets, b->feat_width, b->x_offsets,
                                                             (const double*)b->X, Fp, ksplit, A, B);
    const int kw = 3 * Fp / ksplit;
    const int64_t batch = P * ksplit;
    CUtensorMap ta, tb;
    cudaError_t e = rs_make_tmap_bf16_3d(&ta, A, batch, RS_MAXV, kw, kw, tc::BM);
    if (e == cudaSuccess) e = rs_make_tmap_bf16_3d(&tb, B, batch, RS_MAXV, kw, kw, tile_n);
    if (e != cudaSuccess) return e;
    return tile_n == 32 ? gram_gemm<32>(ta, tb, kw, (int)batch, ksplit, b, K, part, dstatus, st)
                        : gram_gemm<64>(ta, tb, kw, (int)batch, ksplit, b, K, part, dstatus, st);
}
