// K5-K8: the learned surrogate.  An MLP 256 -> 512 -> 512 -> 6 (GELU) maps a standardized
// feature vector straight to the six predicted log speedups (a learned stand-in for the
// tier-2 predictor of Sec. 2).  BF16 weights and activations on the tcgen05 tensor cores,
// FP32 accumulation; FP32 master weights with AdamW.
//
// One training step (a fixed sequence, captured once in a CUDA graph and replayed):
//   stage    rows of X (double) -> BF16 X_s [B][256] and its transpose; labels -> Y_s
//   fwd 1,2  U = X W^T + b (FP32 kept for the backward pass), H = gelu(U) (BF16) and H^T
//   fwd 3    out = H2 W3^T + b3; residual; loss; dO = 2 (out - y) / (6B) (BF16) and dO^T
//   dgrad    dU2 = (dO W3) * gelu'(U2);  dU1 = (dU2 W2) * gelu'(U1)   (BF16, and transposes)
//   wgrad    dW3 = dO^T H2, dW2 = dU2^T H1, dW1 = dU1^T X_s             (FP32)
//   bias     db = row sums of the transposed gradients
//   adamw    master weights, moments, BF16 copies W and W^T for the next step
// Every GEMM is D = A B^T with K-contiguous operands, so the epilogues also write the
// transposed activations that the weight-gradient GEMMs read.
#include <math.h>
#include <string.h>

#include <vector>

#include "tc_gemm.cuh"

namespace {

constexpr int kIn = 256, kHid = 512, kOut = 6, kOutP = 16;   // output rows padded to 16

// ---- blob layout (float offsets) --------------------------------------------------------------
struct Blob {
    static constexpr int64_t nW1 = (int64_t)kHid * kIn, nb1 = kHid, nW2 = (int64_t)kHid * kHid, nb2 = kHid;
    static constexpr int64_t nW3 = (int64_t)kOutP * kHid, nb3 = kOutP;
    static constexpr int64_t nP = nW1 + nb1 + nW2 + nb2 + nW3 + nb3;      // one parameter set
    static constexpr int64_t oW1 = 0, ob1 = oW1 + nW1, oW2 = ob1 + nb1, ob2 = oW2 + nW2, oW3 = ob2 + nb2,
                             ob3 = oW3 + nW3;
    // master | m | v | grad  (FP32), then BF16 copies, then feature stats, then counters
    static constexpr int64_t oM = nP, oV = 2 * nP, oG = 3 * nP;
    static constexpr int64_t oBf = 4 * nP;                                 // in floats
    // BF16 region (in bf16 elements from oBf*2 bytes): W1, W2, W3p, W2t, W3t
    static constexpr int64_t bW1 = 0, bW2 = bW1 + nW1, bW3 = bW2 + nW2, bW2t = bW3 + nW3,
                             bW3t = bW2t + nW2, bEnd = bW3t + (int64_t)kHid * kOutP;
    static constexpr int64_t oStats = oBf + (bEnd + 1) / 2 + 64;           // mean[256], std[256]
    static constexpr int64_t oCount = oStats + 2 * kIn;                    // int step, int t
    static constexpr int64_t nFloats = oCount + 64;
};

// GELU in its tanh form (Hendrycks and Gimpel 2016): gelu(u) = u (1 + tanh(c (u + a u^3))) / 2,
// c = sqrt(2 / pi), a = 0.044715, with the hardware tanh (tanh.approx.f32, relative error
// about 2^-11, below the BF16 rounding of the activations): eight FP32 instructions and one
// special-function instruction, so the epilogue stays near the tensor cores' pace.
constexpr float kGeluC = 0.7978845608028654f;
constexpr float kGeluA = 0.044715f;
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu_f(float u) {
    const float t = tanh_hw(kGeluC * fmaf(kGeluA * u * u, u, u));
    return 0.5f * u * (1.0f + t);
}
// d/du: (1 + t) / 2 + u (1 - t^2) c (1 + 3 a u^2) / 2
__device__ __forceinline__ float gelu_grad_f(float u) {
    const float u2 = u * u;
    const float t = tanh_hw(kGeluC * fmaf(kGeluA * u2, u, u));
    return 0.5f * (1.0f + t) + 0.5f * u * (1.0f - t * t) * kGeluC * fmaf(3.0f * kGeluA, u2, 1.0f);
}

// ---- epilogues ---------------------------------------------------------------------------------
struct EpiHidden {           // U = acc + b (FP32, optional); H = gelu(U) (BF16); H^T (BF16, optional)
    const float* bias;
    float* U;
    __nv_bfloat16* H;
    __nv_bfloat16* Ht;
    int64_t ldt;             // rows of the batch (leading dimension of H^T)
    __device__ void operator()(int row, int col0, const float (&v)[16]) const {
        alignas(16) __nv_bfloat16 hb[16];
        alignas(16) float u[16];
        const float4* b4 = reinterpret_cast<const float4*>(bias + col0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 b = __ldg(b4 + q);
            u[4 * q] = v[4 * q] + b.x;
            u[4 * q + 1] = v[4 * q + 1] + b.y;
            u[4 * q + 2] = v[4 * q + 2] + b.z;
            u[4 * q + 3] = v[4 * q + 3] + b.w;
        }
        if (U) {
            float4* d = reinterpret_cast<float4*>(U + (int64_t)row * kHid + col0);
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = reinterpret_cast<const float4*>(u)[q];
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            hb[i] = __float2bfloat16(gelu_f(u[i]));
            if (Ht) Ht[(int64_t)(col0 + i) * ldt + row] = hb[i];
        }
        uint4* dst = reinterpret_cast<uint4*>(H + (int64_t)row * kHid + col0);
        dst[0] = reinterpret_cast<const uint4*>(hb)[0];
        dst[1] = reinterpret_cast<const uint4*>(hb)[1];
    }
};

struct EpiOutput {           // out = acc + b3; training: residual, loss, dO, dO^T; inference: pred
    const float* bias;
    const float* Y;          // [B][16] (training) or null
    float* loss;             // accumulator (training)
    __nv_bfloat16* dO;       // [B][16]
    __nv_bfloat16* dOt;      // [16][B]
    int64_t ldt;
    float scale;             // 2 / (6 B)
    float* pred;             // [B][6] (inference) or null
    // inference ranking (Sec. 2 tier 3 on the surrogate's predictions), optional
    const uint8_t* masks;    // [B] version masks (candidates: optimizations not applied)
    int flags, k;
    float log_tau;
    uint32_t* rec_code;      // [B]
    double* rec_pred;        // [B][k]
    __device__ void rank_row(int row, const float (&o)[16]) const {
        const int cand = (flags & RS_RANK_ALL) || !masks ? 63 : (~masks[row] & 63);
        int above = 0, bm[kOut];
#pragma unroll
        for (int j = 0; j < kOut; ++j) {
            bm[j] = 0;
            above |= (((cand >> j) & 1) && o[j] >= log_tau) << j;
        }
#pragma unroll
        for (int i = 0; i < kOut; ++i)
#pragma unroll
            for (int j = i + 1; j < kOut; ++j) {
                if (o[i] >= o[j]) bm[j] |= 1 << i;
                else bm[i] |= 1 << j;
            }
        uint32_t code = 0x0FFFFFF0u;
        int c = 0;
        double rp[kOut];
#pragma unroll
        for (int x = 0; x < kOut; ++x) rp[x] = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
        for (int j = 0; j < kOut; ++j) {
            const int pos = __popc(bm[j] & above);
            if (((above >> j) & 1) && pos < k) {
                code = (code & ~(0xFu << (4 + 4 * pos))) | ((uint32_t)j << (4 + 4 * pos));
#pragma unroll
                for (int x = 0; x < kOut; ++x)
                    if (x == pos) rp[x] = o[j];
                ++c;
            }
        }
        rec_code[row] = (code & ~0xFu) | (uint32_t)c;
        if (rec_pred)
#pragma unroll
            for (int x = 0; x < kOut; ++x)
                if (x < k) rec_pred[(int64_t)row * k + x] = rp[x];
    }
    __device__ void operator()(int row, int col0, const float (&v)[16]) const {
        if (col0 != 0) return;
        if (rec_code) {
            float o[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) o[i] = v[i] + bias[i];
            rank_row(row, o);
        }
        float l = 0.f;
        alignas(16) __nv_bfloat16 g[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float out = v[i] + bias[i];
            float d = 0.f;
            if (i < kOut) {
                if (pred) pred[(int64_t)row * kOut + i] = out;
                if (Y) {
                    const float r = out - Y[(int64_t)row * kOutP + i];
                    l += 0.5f * scale * r * r;      // r^2 / (6 B): the minibatch MSE
                    d = scale * r;
                }
            }
            g[i] = __float2bfloat16(d);
            if (dOt) dOt[(int64_t)i * ldt + row] = g[i];
        }
        if (dO) {
            uint4* dst = reinterpret_cast<uint4*>(dO + (int64_t)row * kOutP);
            dst[0] = reinterpret_cast<const uint4*>(g)[0];
            dst[1] = reinterpret_cast<const uint4*>(g)[1];
        }
        if (loss) atomicAdd(loss, l);
    }
};

struct EpiGeluGrad {         // dU = acc * gelu'(U): BF16 dU (optional) and dU^T
    const float* U;
    __nv_bfloat16* dU;
    __nv_bfloat16* dUt;
    int64_t ldt;
    __device__ void operator()(int row, int col0, const float (&v)[16]) const {
        alignas(16) __nv_bfloat16 g[16];
        alignas(16) float u[16];
        const float4* u4 = reinterpret_cast<const float4*>(U + (int64_t)row * kHid + col0);
#pragma unroll
        for (int q = 0; q < 4; ++q) reinterpret_cast<float4*>(u)[q] = u4[q];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            g[i] = __float2bfloat16(v[i] * gelu_grad_f(u[i]));
            dUt[(int64_t)(col0 + i) * ldt + row] = g[i];
        }
        if (dU) {
            uint4* dst = reinterpret_cast<uint4*>(dU + (int64_t)row * kHid + col0);
            dst[0] = reinterpret_cast<const uint4*>(g)[0];
            dst[1] = reinterpret_cast<const uint4*>(g)[1];
        }
    }
};

struct EpiF32Part {          // split-K partial of a weight gradient: slice z -> D + z * zstride
                             // (N, ldd, zstride multiples of 16: whole 16-column chunks)
    float* D;
    int64_t ldd;
    int64_t zstride;
    int N;
    __device__ void operator()(int z, int row, int col0, const float (&v)[16]) const {
        float4* d = reinterpret_cast<float4*>(D + (int64_t)z * zstride + (int64_t)row * ldd + col0);
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
};

struct EpiF32 {              // plain FP32 store (weight gradients; N, ldd multiples of 16)
    float* D;
    int64_t ldd;
    int N;
    __device__ void operator()(int row, int col0, const float (&v)[16]) const {
        float4* d = reinterpret_cast<float4*>(D + (int64_t)row * ldd + col0);
#pragma unroll
        for (int q = 0; q < 4; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
};

// Pipeline depth of the persistent GEMM (one CTA per SM): four 32 KB stages (BN = 128).
constexpr int kStages = 4;

template <int BN, int S, class Epi>
cudaError_t gemm_attr();

template <int BN, class Epi, bool BATCHED = false>
cudaError_t gemm_attr() {
    return cudaFuncSetAttribute(tc::gemm_kernel<BN, kStages, Epi, BATCHED>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, tc::Layout<BN, kStages>::kBytes);
}

// The function attributes of every product of a training step, set before a graph capture.
cudaError_t all_attrs() {
    cudaError_t e = gemm_attr<128, EpiHidden>();
    if (e == cudaSuccess) e = gemm_attr<32, EpiOutput>();
    if (e == cudaSuccess) e = gemm_attr<128, EpiGeluGrad>();
    if (e == cudaSuccess) e = gemm_attr<128, EpiF32>();
    if (e == cudaSuccess) e = gemm_attr<128, EpiF32Part, true>();
    return e;
}

// Split-K product over `slices` K ranges (rank-3 maps from rs_make_tmap_bf16_kslices): batch z
// is range z; the epilogue gets z.
template <int BN, class Epi>
cudaError_t gemm_slices(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int Kslice, int slices,
                        const Epi& epi, int* err, cudaStream_t st) {
    return tc::gemm_launch<BN, kStages, Epi, true>(ta, tb, M, N, Kslice, slices, epi, err, st);
}

template <int BN, class Epi>
cudaError_t gemm(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, const Epi& epi, int* err,
                 cudaStream_t st) {
    return tc::gemm_launch<BN, kStages, Epi>(ta, tb, M, N, K, 1, epi, err, st);
}

// ---- small kernels -----------------------------------------------------------------------------
// Stage a minibatch: rows (r0 + i) mod n of X (double [n][256]) -> BF16 X_s and X_s^T, labels
// (double [n][6], NaN treated as 0 with zero weight) -> Y_s [B][16].  r0 = step * B, with the
// step read from the device counter so the same launch serves every step of a graph.
__global__ void __launch_bounds__(256)
stage_kernel(const double* __restrict__ X, const double* __restrict__ Yin, int64_t n, int B, const int* step,
             int64_t fixed_r0, __nv_bfloat16* Xs, __nv_bfloat16* Xt, float* Ys) {
    const int64_t r0 = step ? (int64_t)(*step) * B : fixed_r0;
    const int i = blockIdx.x;                   // batch row
    if (i >= B) return;
    const int64_t src = (r0 + i) % n;
    for (int f = threadIdx.x; f < kIn; f += blockDim.x) {
        const __nv_bfloat16 v = __float2bfloat16((float)X[src * kIn + f]);
        Xs[(int64_t)i * kIn + f] = v;
        if (Xt) Xt[(int64_t)f * B + i] = v;
    }
    if (Ys && threadIdx.x < kOutP) {
        float y = 0.f;
        if (threadIdx.x < kOut) {
            const double d = Yin[src * kOut + threadIdx.x];
            y = isfinite(d) ? (float)d : 0.f;
        }
        Ys[(int64_t)i * kOutP + threadIdx.x] = y;
    }
}

// double -> BF16 and double -> float with integer operations only (this part's double
// conversions run on its narrow FP64 pipe).  BF16: round to nearest, ties to even, on the 52
// fraction bits; float: truncated fraction (used for the OOD score).  Values outside the
// normal float range take the conversion instructions.
__device__ __forceinline__ bool f32_normal_range(long long b) {
    const int e = (int)((b >> 52) & 0x7ff);
    return e > 1023 - 126 && e < 1023 + 127;
}
__device__ __forceinline__ __nv_bfloat16 bf16_of(double x) {
    const long long b = __double_as_longlong(x);
    if (!f32_normal_range(b)) return __float2bfloat16((float)x);
    const unsigned long long u = (unsigned long long)b;
    // keep 7 fraction bits: round on bit 45, ties to even on bit 45 of the kept part
    const unsigned long long r = u + ((1ull << 44) - 1ull) + ((u >> 45) & 1ull);
    const unsigned long long m = (r >> 45) & 0x7full;                // 7 fraction bits
    const int e = (int)((r >> 52) & 0x7ff) - 1023 + 127;             // carry may bump the exponent
    const unsigned short h = (unsigned short)(((u >> 63) << 15) | ((unsigned)e << 7) | (unsigned)m);
    return __ushort_as_bfloat16(h);
}
__device__ __forceinline__ float f32_trunc_of(double x) {
    const long long b = __double_as_longlong(x);
    if (!f32_normal_range(b)) return (float)x;
    const unsigned long long u = (unsigned long long)b;
    const unsigned e = (unsigned)((u >> 52) & 0x7ff) - 1023u + 127u;
    return __uint_as_float((unsigned)((u >> 63) << 31) | (e << 23) | (unsigned)((u >> 29) & 0x7fffff));
}

// Inference staging: rows of X (double [n][256]) -> BF16 X_s, one warp per row (lane l takes
// features 8l .. 8l+7: 64 contiguous bytes in, 16 out), grid-stride over the chunk; with the
// training statistics given, the same pass forms the out-of-distribution score (mean over
// features of ((x - mean) / sd)^2, FP32) and the fallback flag of each row.
__global__ void __launch_bounds__(256)
infer_stage_kernel(const double* __restrict__ X, int64_t B, __nv_bfloat16* Xs, const float* __restrict__ mean,
                   const float* __restrict__ sd, float thr, float* score, uint8_t* fallback) {
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    float mu[8], sinv[8];                    // per feature: mean and 1 / sd (0 where sd = 0)
    if (mean) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            mu[e] = mean[8 * lane + e];
            const float d = sd[8 * lane + e];
            sinv[e] = d > 0.f ? 1.0f / d : 0.f;
        }
    }
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < B; r += wstride) {
        const double2* src = reinterpret_cast<const double2*>(X + r * kIn + 8 * lane);
        double x[8];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const double2 v = __ldcs(src + e);       // read once: streaming
            x[2 * e] = v.x;
            x[2 * e + 1] = v.y;
        }
        alignas(16) __nv_bfloat16 hb[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) hb[e] = bf16_of(x[e]);
        *reinterpret_cast<uint4*>(Xs + r * kIn + 8 * lane) = *reinterpret_cast<const uint4*>(hb);
        if (mean) {
            float s = 0.f;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float d = (f32_trunc_of(x[e]) - mu[e]) * sinv[e];
                s = fmaf(d, d, s);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                s /= kIn;
                if (score) score[r] = s;
                if (fallback) fallback[r] = s > thr ? 1 : 0;
            }
        }
    }
}

// Row sums of a transposed gradient [rows][B] (BF16) -> FP32 bias gradient; one warp per row.
__global__ void __launch_bounds__(256)
rowsum_kernel(const __nv_bfloat16* __restrict__ T, int rows, int B, float* out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= rows) return;
    float s = 0.f;
    for (int i = lane; i < B; i += 32) s += __bfloat162float(T[(int64_t)w * B + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[w] = s;
}

// Sum of the split-K partials of the three weight gradients, slice 0 first (a fixed order,
// so every step and every graph replay adds the same numbers the same way).  The partials
// of one slice are laid out [W1 | W2 | W3] (nW1 + nW2 + nW3 floats).
__global__ void __launch_bounds__(256)
reduce_wgrad_kernel(const float* __restrict__ part, int slices, float* G) {
    constexpr int64_t n = Blob::nW1 + Blob::nW2 + Blob::nW3;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int z = 0; z < slices; ++z) s += part[(int64_t)z * n + i];
    const int64_t o = i < Blob::nW1 ? Blob::oW1 + i
                    : i < Blob::nW1 + Blob::nW2 ? Blob::oW2 + (i - Blob::nW1)
                                                : Blob::oW3 + (i - Blob::nW1 - Blob::nW2);
    G[o] = s;
}

// BF16 copies of the master weights: W1, W2, W3 (padded rows) and the transposes W2^T, W3^T.
__global__ void __launch_bounds__(256)
sync_bf16_kernel(const float* __restrict__ P, __nv_bfloat16* bf) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Blob::nW1) bf[Blob::bW1 + i] = __float2bfloat16(P[Blob::oW1 + i]);
    if (i < Blob::nW2) {
        const float w = P[Blob::oW2 + i];
        bf[Blob::bW2 + i] = __float2bfloat16(w);
        const int64_t r = i / kHid, c = i % kHid;
        bf[Blob::bW2t + c * kHid + r] = __float2bfloat16(w);
    }
    if (i < Blob::nW3) {
        const int64_t r = i / kHid, c = i % kHid;           // r < 16 (rows >= 6 stay zero)
        const float w = r < kOut ? P[Blob::oW3 + i] : 0.f;
        bf[Blob::bW3 + i] = __float2bfloat16(w);
        bf[Blob::bW3t + c * kOutP + r] = __float2bfloat16(w);
    }
}

// AdamW over every parameter (padded output rows keep zero gradient and stay zero).
__global__ void __launch_bounds__(256)
adamw_kernel(float* blob, float lr, float b1, float b2, float eps, float wd, int* counters) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int t = counters[1] + 1;              // this step's index (1-based)
    if (i < Blob::nP) {
        float* P = blob;
        float* m = blob + Blob::oM;
        float* v = blob + Blob::oV;
        const float g = blob[Blob::oG + i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / (1.f - powf(b1, (float)t));
        const float vh = vi / (1.f - powf(b2, (float)t));
        P[i] = P[i] - lr * (mh / (sqrtf(vh) + eps) + wd * P[i]);
    }
}

// A call continues from the blob's counters (a restored checkpoint resumes the same sequence
// of minibatches and Adam steps); the minibatch position wraps into this call's rows.
__global__ void wrap_counters_kernel(int* counters, int64_t steps_per_epoch) {
    int64_t q = counters[0] % steps_per_epoch;
    if (q < 0) q += steps_per_epoch;                         // (a blob not zeroed by its owner)
    counters[0] = (int)q;
    if (counters[1] < 0) counters[1] = 0;
}
__global__ void bump_counters_kernel(int* counters, int64_t steps_per_epoch) {
    counters[1] += 1;                                        // Adam t
    counters[0] = (int)((counters[0] + 1) % steps_per_epoch); // minibatch index
}

// Feature mean / std over the training rows (for the out-of-distribution score): each
// block sums a strided set of rows with one thread per feature (coalesced), then adds its
// partial sums into acc[2][256] (double); feature_stats_finish turns them into mean / std.
__global__ void __launch_bounds__(kIn)
feature_stats_kernel(const double* __restrict__ X, int64_t n, double* acc) {
    const int f = threadIdx.x;
    double s = 0.0, q = 0.0;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const double x = X[r * kIn + f];
        s += x;
        q += x * x;
    }
    atomicAdd(acc + f, s);
    atomicAdd(acc + kIn + f, q);
}
__global__ void feature_stats_finish(const double* acc, int64_t n, float* mean, float* sd) {
    const int f = threadIdx.x;
    const double m = acc[f] / n;
    mean[f] = (float)m;
    sd[f] = (float)sqrt(fmax(acc[kIn + f] / n - m * m, 0.0));
}

// ---- training workspace --------------------------------------------------------------------------
struct TrainWs {
    __nv_bfloat16 *Xs, *Xt, *H1, *H1t, *H2, *H2t, *dO, *dOt, *dU2, *dU2t, *dU1t;
    float *Ys, *U1, *U2;
    double* stats_acc;
    float* part;              // split-K partials of the weight gradients (slices > 1)
    int slices;
    size_t bytes;
};

// K ranges of the weight-gradient products (K = the minibatch rows): the largest power of two
// up to 16 that leaves at least 256 rows per range in whole 64-row blocks.  A few output tiles
// then spread over up to 16x as many CTAs.
int wgrad_slices(int B) {
    int s = 1;
    while (s < 16 && B % (64 * 2 * s) == 0 && B / (2 * s) >= 256) s *= 2;
    return s;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

TrainWs carve_train(void* base, int B) {
    TrainWs w{};
    char* c = (char*)base;
    size_t o = 0;
    auto take = [&](size_t b) { char* p = c ? c + o : nullptr; o += a256(b); return p; };
    const size_t bf = sizeof(__nv_bfloat16);
    w.Xs = (__nv_bfloat16*)take((size_t)B * kIn * bf);
    w.Xt = (__nv_bfloat16*)take((size_t)B * kIn * bf);
    w.H1 = (__nv_bfloat16*)take((size_t)B * kHid * bf);
    w.H1t = (__nv_bfloat16*)take((size_t)B * kHid * bf);
    w.H2 = (__nv_bfloat16*)take((size_t)B * kHid * bf);
    w.H2t = (__nv_bfloat16*)take((size_t)B * kHid * bf);
    w.dO = (__nv_bfloat16*)take((size_t)B * kOutP * bf);
    w.dOt = (__nv_bfloat16*)take((size_t)B * kOutP * bf);
    w.dU2 = (__nv_bfloat16*)take((size_t)B * kHid * bf);
    w.dU2t = (__nv_bfloat16*)take((size_t)B * kHid * bf);
    w.dU1t = (__nv_bfloat16*)take((size_t)B * kHid * bf);
    w.Ys = (float*)take((size_t)B * kOutP * sizeof(float));
    w.U1 = (float*)take((size_t)B * kHid * sizeof(float));
    w.U2 = (float*)take((size_t)B * kHid * sizeof(float));
    w.stats_acc = (double*)take(2 * kIn * sizeof(double));
    w.slices = wgrad_slices(B);
    w.part = w.slices > 1 ? (float*)take((size_t)w.slices * (Blob::nW1 + Blob::nW2 + Blob::nW3) * sizeof(float))
                          : nullptr;
    w.bytes = o;
    return w;
}

struct Maps {
    CUtensorMap Xs, W1, H1, W2, H2, W3, dO, W3t, dU2, W2t, dOt, H2t, dU2t, H1t, dU1t, Xt;
    // split-K views of the transposed operands of the weight gradients (slices > 1)
    CUtensorMap sdOt, sH2t, sdU2t, sH1t, sdU1t, sXt;
};

cudaError_t make_maps(Maps& m, const TrainWs& w, const __nv_bfloat16* bf, int B) {
    cudaError_t e = cudaSuccess;
    auto mk = [&](CUtensorMap* t, const void* p, int64_t rows, int64_t cols, int box) {
        if (e == cudaSuccess) e = rs_make_tmap_bf16(t, p, rows, cols, cols, box);
    };
    mk(&m.Xs, w.Xs, B, kIn, 128);
    mk(&m.W1, bf + Blob::bW1, kHid, kIn, 128);
    mk(&m.H1, w.H1, B, kHid, 128);
    mk(&m.W2, bf + Blob::bW2, kHid, kHid, 128);
    mk(&m.H2, w.H2, B, kHid, 128);
    mk(&m.W3, bf + Blob::bW3, kOutP, kHid, 32);
    mk(&m.dO, w.dO, B, kOutP, 128);
    mk(&m.W3t, bf + Blob::bW3t, kHid, kOutP, 128);
    mk(&m.dU2, w.dU2, B, kHid, 128);
    mk(&m.W2t, bf + Blob::bW2t, kHid, kHid, 128);
    mk(&m.dOt, w.dOt, kOutP, B, 128);
    mk(&m.H2t, w.H2t, kHid, B, 128);
    mk(&m.dU2t, w.dU2t, kHid, B, 128);
    mk(&m.H1t, w.H1t, kHid, B, 128);
    mk(&m.dU1t, w.dU1t, kHid, B, 128);
    mk(&m.Xt, w.Xt, kIn, B, 128);
    if (w.slices > 1) {
        auto ks = [&](CUtensorMap* t, const void* p, int64_t rows, int box) {
            if (e == cudaSuccess) e = rs_make_tmap_bf16_kslices(t, p, rows, B, B, w.slices, box);
        };
        ks(&m.sdOt, w.dOt, kOutP, 128);
        ks(&m.sH2t, w.H2t, kHid, 128);
        ks(&m.sdU2t, w.dU2t, kHid, 128);
        ks(&m.sH1t, w.H1t, kHid, 128);
        ks(&m.sdU1t, w.dU1t, kHid, 128);
        ks(&m.sXt, w.Xt, kIn, 128);
    }
    return e;
}

// Forward + backward for the staged minibatch: gradients into the blob's grad region.
cudaError_t step_body(float* blob, const TrainWs& w, const Maps& m, int B, float* loss_slot, int* err,
                      cudaStream_t st) {
    float* G = blob + Blob::oG;
    const float* P = blob;
    cudaError_t e;
    const float sc = 2.0f / (6.0f * (float)B);
    e = gemm<128>(m.Xs, m.W1, B, kHid, kIn, EpiHidden{P + Blob::ob1, w.U1, w.H1, w.H1t, B}, err, st);
    if (e == cudaSuccess)
        e = gemm<128>(m.H1, m.W2, B, kHid, kHid, EpiHidden{P + Blob::ob2, w.U2, w.H2, w.H2t, B}, err, st);
    if (e == cudaSuccess)
        e = gemm<32>(m.H2, m.W3, B, kOutP, kHid,
                     EpiOutput{P + Blob::ob3, w.Ys, loss_slot, w.dO, w.dOt, B, sc, nullptr, nullptr, 0, 0, 0.f,
                               nullptr, nullptr}, err, st);
    if (e == cudaSuccess)      // dU2 = (dO W3) * gelu'(U2)
        e = gemm<128>(m.dO, m.W3t, B, kHid, kOutP, EpiGeluGrad{w.U2, w.dU2, w.dU2t, B}, err, st);
    if (e == cudaSuccess)      // dU1 = (dU2 W2) * gelu'(U1)
        e = gemm<128>(m.dU2, m.W2t, B, kHid, kHid, EpiGeluGrad{w.U1, nullptr, w.dU1t, B}, err, st);
    if (w.slices > 1) {        // weight gradients split over K ranges, then summed in order
        constexpr int64_t nPart = Blob::nW1 + Blob::nW2 + Blob::nW3;
        const int S = w.slices, ks = B / S;
        if (e == cudaSuccess)  // dW3 = dO^T H2
            e = gemm_slices<128>(m.sdOt, m.sH2t, kOutP, kHid, ks, S,
                                                EpiF32Part{w.part + Blob::nW1 + Blob::nW2, kHid, nPart, kHid}, err, st);
        if (e == cudaSuccess)  // dW2 = dU2^T H1
            e = gemm_slices<128>(m.sdU2t, m.sH1t, kHid, kHid, ks, S,
                                                EpiF32Part{w.part + Blob::nW1, kHid, nPart, kHid}, err, st);
        if (e == cudaSuccess)  // dW1 = dU1^T X
            e = gemm_slices<128>(m.sdU1t, m.sXt, kHid, kIn, ks, S,
                                                EpiF32Part{w.part, kIn, nPart, kIn}, err, st);
        if (e == cudaSuccess) {
            reduce_wgrad_kernel<<<(unsigned)((nPart + 255) / 256), 256, 0, st>>>(w.part, S, G);
            e = cudaGetLastError();
        }
    } else {
        if (e == cudaSuccess)  // dW3 = dO^T H2
            e = gemm<128>(m.dOt, m.H2t, kOutP, kHid, B, EpiF32{G + Blob::oW3, kHid, kHid}, err, st);
        if (e == cudaSuccess)  // dW2 = dU2^T H1
            e = gemm<128>(m.dU2t, m.H1t, kHid, kHid, B, EpiF32{G + Blob::oW2, kHid, kHid}, err, st);
        if (e == cudaSuccess)  // dW1 = dU1^T X
            e = gemm<128>(m.dU1t, m.Xt, kHid, kIn, B, EpiF32{G + Blob::oW1, kIn, kIn}, err, st);
    }
    if (e == cudaSuccess) {
        rowsum_kernel<<<(kOut * 32 + 255) / 256, 256, 0, st>>>(w.dOt, kOut, B, G + Blob::ob3);
        rowsum_kernel<<<(kHid * 32 + 255) / 256, 256, 0, st>>>(w.dU2t, kHid, B, G + Blob::ob2);
        rowsum_kernel<<<(kHid * 32 + 255) / 256, 256, 0, st>>>(w.dU1t, kHid, B, G + Blob::ob1);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

size_t rs_surrogate_blob_floats() { return (size_t)Blob::nFloats; }
size_t rs_surrogate_train_ws_bytes(int B) { return carve_train(nullptr, B).bytes; }
size_t rs_surrogate_infer_ws_bytes(int64_t chunk) {
    return a256((size_t)chunk * kIn * 2) + 2 * a256((size_t)chunk * kHid * 2);
}
int64_t rs_surrogate_blob_offset(int which) {
    switch (which) {
        case 0: return Blob::oW1;
        case 1: return Blob::ob1;
        case 2: return Blob::oW2;
        case 3: return Blob::ob2;
        case 4: return Blob::oW3;
        case 5: return Blob::ob3;
        case 6: return Blob::oM;
        case 7: return Blob::oV;
        case 8: return Blob::oG;
        case 9: return Blob::oStats;
        case 10: return Blob::oCount;
        default: return -1;
    }
}

// Train for `steps` minibatches of B rows; rows are taken in order (wrapping) from X / Y.
// graph != 0: the step is captured once and replayed.
cudaError_t rs_launch_surrogate_train(float* blob, const double* X, const double* Y, int64_t n, int B,
                                      int64_t steps, float lr, float wd, float* loss_curve, void* ws,
                                      int use_graph, int* err, cudaStream_t st) {
    TrainWs w = carve_train(ws, B);
    __nv_bfloat16* bf = reinterpret_cast<__nv_bfloat16*>(blob + Blob::oBf);
    int* counters = reinterpret_cast<int*>(blob + Blob::oCount);
    Maps m;
    cudaError_t e = make_maps(m, w, bf, B);
    if (e == cudaSuccess) e = all_attrs();
    if (e != cudaSuccess) return e;
    const int64_t spe = n / B > 0 ? n / B : 1;
    // statistics for the OOD score, BF16 copies of the initial weights, the counters' position
    e = cudaMemsetAsync(w.stats_acc, 0, 2 * kIn * sizeof(double), st);
    if (e != cudaSuccess) return e;
    feature_stats_kernel<<<(unsigned)(n < 1024 ? n : 1024), kIn, 0, st>>>(X, n, w.stats_acc);
    feature_stats_finish<<<1, kIn, 0, st>>>(w.stats_acc, n, blob + Blob::oStats, blob + Blob::oStats + kIn);
    sync_bf16_kernel<<<(unsigned)((Blob::nW2 + 255) / 256), 256, 0, st>>>(blob, bf);
    wrap_counters_kernel<<<1, 1, 0, st>>>(counters, spe);
    e = cudaGetLastError();
    if (e == cudaSuccess && loss_curve) e = cudaMemsetAsync(loss_curve, 0, steps * sizeof(float), st);
    if (e != cudaSuccess) return e;
    // one step; the loss goes to loss_curve[t - 1] through a device-side pointer bump
    float* loss_dev = nullptr;     // loss slot is chosen per step below
    auto one_step = [&](int64_t s, cudaStream_t q) -> cudaError_t {
        stage_kernel<<<B, 256, 0, q>>>(X, Y, n, B, counters, 0, w.Xs, w.Xt, w.Ys);
        cudaError_t e2 = step_body(blob, w, m, B, loss_curve ? loss_curve + s : loss_dev, err, q);
        if (e2 != cudaSuccess) return e2;
        adamw_kernel<<<(unsigned)((Blob::nP + 255) / 256), 256, 0, q>>>(blob, lr, 0.9f, 0.999f, 1e-8f, wd, counters);
        sync_bf16_kernel<<<(unsigned)((Blob::nW2 + 255) / 256), 256, 0, q>>>(blob, bf);
        bump_counters_kernel<<<1, 1, 0, q>>>(counters, spe);
        return cudaGetLastError();
    };
    if (!use_graph || !loss_curve) {
        for (int64_t s = 0; s < steps && e == cudaSuccess; ++s) e = one_step(s, st);
        return e;
    }
    // The loss slot differs per step, so capture one graph per distinct slot would defeat the
    // purpose: capture with the slot of step 0 and accumulate into a scratch float that a tiny
    // copy kernel moves to loss_curve[s] after each replay.
    float* slot = blob + Blob::oCount + 8;
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t eb = cudaMemsetAsync(slot, 0, sizeof(float), cap);
        stage_kernel<<<B, 256, 0, cap>>>(X, Y, n, B, counters, 0, w.Xs, w.Xt, w.Ys);
        if (eb == cudaSuccess) eb = step_body(blob, w, m, B, slot, err, cap);
        adamw_kernel<<<(unsigned)((Blob::nP + 255) / 256), 256, 0, cap>>>(blob, lr, 0.9f, 0.999f, 1e-8f, wd, counters);
        sync_bf16_kernel<<<(unsigned)((Blob::nW2 + 255) / 256), 256, 0, cap>>>(blob, bf);
        bump_counters_kernel<<<1, 1, 0, cap>>>(counters, spe);
        e = cudaStreamEndCapture(cap, &g);
        if (eb != cudaSuccess) e = eb;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    cudaEvent_t ev;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        // order the graph after the setup work on st
        cudaEventRecord(ev, st);
        cudaStreamWaitEvent(cap, ev, 0);
        for (int64_t s = 0; s < steps && e == cudaSuccess; ++s) {
            e = cudaGraphLaunch(ge, cap);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(loss_curve + s, slot, sizeof(float), cudaMemcpyDeviceToDevice, cap);
        }
        cudaEventRecord(ev, cap);
        cudaStreamWaitEvent(st, ev, 0);
        cudaEventDestroy(ev);
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    return e;
}

// Forward pass over n rows in chunks: pred [n][6] (FP32); optional OOD score and fallback flags.
cudaError_t rs_launch_surrogate_infer(const float* blob, const double* X, int64_t n, float ood_thr,
                                      float* pred, float* score, uint8_t* fallback, const uint8_t* masks,
                                      int k, double tau, int flags, uint32_t* rec_code, double* rec_pred,
                                      void* ws, int64_t chunk, int* err, cudaStream_t st) {
    const __nv_bfloat16* bf = reinterpret_cast<const __nv_bfloat16*>(blob + Blob::oBf);
    char* c = (char*)ws;
    __nv_bfloat16* Xs = (__nv_bfloat16*)c;
    __nv_bfloat16* H1 = (__nv_bfloat16*)(c + a256((size_t)chunk * kIn * 2));
    __nv_bfloat16* H2 = (__nv_bfloat16*)(c + a256((size_t)chunk * kIn * 2) + a256((size_t)chunk * kHid * 2));
    cudaError_t e = cudaSuccess;
    for (int64_t r0 = 0; r0 < n && e == cudaSuccess; r0 += chunk) {
        const int B = (int)((n - r0) < chunk ? (n - r0) : chunk);
        CUtensorMap tX, tW1, tH1, tW2, tH2, tW3;
        e = rs_make_tmap_bf16(&tX, Xs, B, kIn, kIn, 128);
        if (e == cudaSuccess) e = rs_make_tmap_bf16(&tW1, bf + Blob::bW1, kHid, kIn, kIn, 128);
        if (e == cudaSuccess) e = rs_make_tmap_bf16(&tH1, H1, B, kHid, kHid, 128);
        if (e == cudaSuccess) e = rs_make_tmap_bf16(&tW2, bf + Blob::bW2, kHid, kHid, kHid, 128);
        if (e == cudaSuccess) e = rs_make_tmap_bf16(&tH2, H2, B, kHid, kHid, 128);
        if (e == cudaSuccess) e = rs_make_tmap_bf16(&tW3, bf + Blob::bW3, kOutP, kHid, kHid, 32);
        if (e != cudaSuccess) break;
        const bool ood = score || fallback;
        const int sblocks = (int)((B + 7) / 8) < 4096 ? (int)((B + 7) / 8) : 4096;
        infer_stage_kernel<<<sblocks, 256, 0, st>>>(X + r0 * kIn, B, Xs, ood ? blob + Blob::oStats : nullptr,
                                                     blob + Blob::oStats + kIn, ood_thr,
                                                     score ? score + r0 : nullptr,
                                                     fallback ? fallback + r0 : nullptr);
        e = gemm<128>(tX, tW1, B, kHid, kIn, EpiHidden{blob + Blob::ob1, nullptr, H1, nullptr, B}, err, st);
        if (e == cudaSuccess)
            e = gemm<128>(tH1, tW2, B, kHid, kHid, EpiHidden{blob + Blob::ob2, nullptr, H2, nullptr, B}, err, st);
        if (e == cudaSuccess)
            e = gemm<32>(tH2, tW3, B, kOutP, kHid,
                         EpiOutput{blob + Blob::ob3, nullptr, nullptr, nullptr, nullptr, B, 0.f,
                                   pred ? pred + r0 * kOut : nullptr, masks ? masks + r0 : nullptr, flags, k,
                                   (float)log(tau), rec_code ? rec_code + r0 : nullptr,
                                   rec_pred ? rec_pred + r0 * k : nullptr},
                         err, st);
    }
    return e;
}
