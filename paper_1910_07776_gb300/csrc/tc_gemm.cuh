// tc_gemm.cuh -- BF16 GEMM on the sm_103a tensor cores (tcgen05), used by the surrogate's
// forward / backward kernels, the tensor-core Gram and rs_gemm_bf16.
//
//   D[M][N] (FP32, in tensor memory) = A[M][K] * B[N][K]^T,  A, B BF16, both K-contiguous.
//
// Persistent CTAs (one per SM) walk the 128 x BN output tiles; inside a CTA a TMA producer
// warp, a single-thread MMA issuer and eight epilogue warps run concurrently, connected by
// mbarriers (stage full / empty, accumulator full / empty), with two tensor-memory
// accumulators so that a tile's epilogue overlaps the next tile's MMAs (see gemm_kernel).
// Every mbarrier wait is bounded (1 s of %globaltimer); a wait that gives up sets
// RS_ETIMEOUT in the device status word and the CTA winds down without hanging.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mbar.cuh"
#include "rs_internal.cuh"

namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;                       // one 128-byte swizzle row of BF16
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(dst), "l"((unsigned long long)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
// 3-D tile load: x = K coordinate, y = row within the matrix, z = batch index.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(dst), "l"((unsigned long long)map), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// D(tmem) (+)= A(smem desc) * B(smem desc)^T, kind::f16 (BF16 inputs, FP32 accumulate).
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// 32 lanes x 16 consecutive 32-bit columns: thread i of the warp gets row (lane base + i).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// The same load without the wait: several can be in flight before one tmem_wait_ld().
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile stored in the 128-byte swizzle layout
// (rows of 64 BF16 = 128 B, 8-row groups 1024 B apart), as written by a TMA load with
// CU_TENSOR_MAP_SWIZZLE_128B into a 1024-byte aligned buffer.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused here)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)2 << 61;                           // 128-byte swizzle
    return d;
}
// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int BN, int STAGES>
struct Layout {
    static constexpr int kA = BM * BK * 2;           // bytes of one A stage
    static constexpr int kB = BN * BK * 2;           // bytes of one B stage
    static constexpr int kStage = kA + kB;
    static constexpr int kBars = 1024;               // barrier area after the stages
    static constexpr int kBytes = STAGES * kStage + kBars + 1024;   // + alignment slack
};

constexpr int kEpiWarps = 8;                          // two per TMEM lane quarter
constexpr int kGemmThreads = (2 + kEpiWarps) * 32;    // producer, MMA issuer, epilogue

// Persistent, warp-specialised GEMM over all 128 x BN output tiles of all batches (tile t of
// the CTA's static round-robin: t = blockIdx.x, + gridDim.x, ...; N-blocks fastest, so the
// CTAs working at the same time share their A tiles -- the large, streamed operand -- in L2
// and each is read from DRAM once; the B operands here are weights, L2-resident).
//   warp 0 (one thread): TMA producer -- a STAGES-deep shared-memory ring of 128 x 64 A and
//     BN x 64 B slices (128-byte swizzle) running ahead across tile boundaries;
//   warp 1 (one thread): MMA issuer -- tcgen05.mma (M = 128, N = BN, K = 16) into one of two
//     tensor-memory accumulators, tcgen05.commit frees each stage and, after a tile's last
//     k-block, hands the accumulator to the epilogue;
//   warps 2..9: epilogue -- warp w reads TMEM lane quarter (w mod 4) (rows 32 (w mod 4) ..+31),
//     half of the columns each, 16 at a time with tcgen05.ld, calls the epilogue functor and
//     returns the accumulator to the MMA issuer.
// Two accumulators let a tile's epilogue overlap the next tile's MMAs; the CTA's set-up
// (barriers, tensor-memory allocation) is paid once.  Every mbarrier wait is bounded (1 s);
// a wait that gives up sets RS_ETIMEOUT, the role leaves its loop, the producer waits
// (bounded) for its loads still in flight, and the CTA frees its tensor memory and returns.
// Epi: __device__ void operator()(int row, int col0, const float (&v)[16]) const, called for
// every row < M with the 16 accumulator columns starting at col0 (col0 < N).  BATCHED: the
// operands are rank-3 tensor maps [batch][rows][K] and the functor is called as
// epi(z, row, col0, v).
template <int BN, int STAGES, class Epi, bool BATCHED = false>
__global__ void __launch_bounds__(kGemmThreads, 1)
gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N,
            int K, int batch, Epi epi, int* err) {
    using L = Layout<BN, STAGES>;
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256 && (BN & (BN - 1)) == 0, "BN: 32..256, power of 2");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    // barriers: full[S], empty[S], tfull[2], tempty[2], drain; then the tensor-memory slot
    const uint32_t bars = base + STAGES * L::kStage;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + STAGES * L::kStage + 8 * (2 * STAGES + 5));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (STAGES + s); };
    auto tfull = [&](int a) { return bars + 8u * (2 * STAGES + a); };
    auto tempty = [&](int a) { return bars + 8u * (2 * STAGES + 2 + a); };
    const uint32_t drain = bars + 8u * (2 * STAGES + 4);
    const int mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
    const long long tiles = (long long)mt * nt * batch;
    const int nk = (K + BK - 1) / BK;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull(a), 1);
            mbar_init(tempty(a), kEpiWarps);
        }
        mbar_init(drain, 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), 2 * BN);
        tmem_relinquish();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {                             // ---- TMA producer
            long long kg = 0;                        // k-blocks issued by this CTA
            bool ok = true;
            for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                const int z = (int)(t / ((long long)mt * nt));
                const int rem = (int)(t - (long long)z * mt * nt);
                const int m0 = (rem / nt) * BM, n0 = (rem % nt) * BN;
                for (int kb = 0; kb < nk; ++kb, ++kg) {
                    const int s = (int)(kg % STAGES);
                    const long long j = kg / STAGES;
                    if (j >= 1 && !mbar_wait(empty(s), (uint32_t)((j - 1) & 1), err, 11)) {
                        ok = false;
                        break;
                    }
                    const uint32_t a = base + s * L::kStage, b = a + L::kA;
                    mbar_expect_tx(full(s), L::kStage);
                    if (BATCHED) {
                        tma_load_3d(a, &ta, full(s), kb * BK, m0, z);
                        tma_load_3d(b, &tb, full(s), kb * BK, n0, z);
                    } else {
                        tma_load_2d(a, &ta, full(s), kb * BK, m0);
                        tma_load_2d(b, &tb, full(s), kb * BK, n0);
                    }
                }
            }
            if (!ok)   // wait (bounded) for this CTA's loads that may still be in flight
                for (long long q = kg - STAGES < 0 ? 0 : kg - STAGES; q < kg; ++q)
                    mbar_wait(full((int)(q % STAGES)), (uint32_t)((q / STAGES) & 1), err, 12);
        }
    } else if (warp == 1) {
        if (lane == 0) {                             // ---- MMA issuer
            const uint32_t idesc = idesc_bf16(BM, BN);
            long long kg = 0;
            int tl = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++tl) {
                const int acc = tl & 1, u = tl >> 1;
                if (u >= 1 && !mbar_wait(tempty(acc), (uint32_t)((u - 1) & 1), err, 13)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * BN);
                for (int kb = 0; kb < nk; ++kb, ++kg) {
                    const int s = (int)(kg % STAGES);
                    if (!mbar_wait(full(s), (uint32_t)((kg / STAGES) & 1), err, 14)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t a = base + s * L::kStage, b = a + L::kA;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk)
                        mma_bf16(d, sw128_desc(a + kk * 32), sw128_desc(b + kk * 32), idesc, (kb | kk) != 0);
                    mma_commit(empty(s));
                }
                if (ok) mma_commit(tfull(acc));
            }
            // every MMA this thread issued has completed before the tensor memory is freed
            mma_commit(drain);
            mbar_wait(drain, 0, err, 16);
        }
    } else {                                         // ---- epilogue
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        int tl = 0;
        for (long long t = blockIdx.x; t < tiles; t += gridDim.x, ++tl) {
            const int acc = tl & 1, u = tl >> 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(tfull(acc), (uint32_t)(u & 1), err, 15) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            fence_after();
            const int z = (int)(t / ((long long)mt * nt));
            const int rem = (int)(t - (long long)z * mt * nt);
            const int m0 = (rem / nt) * BM, n0 = (rem % nt) * BN;
            const int row = m0 + quarter * 32 + lane;
            const uint32_t trow = tmem + (uint32_t)(acc * BN) + ((uint32_t)(quarter * 32) << 16);
            // this warp's columns: all their tensor-memory loads in flight, then one wait
            constexpr int kChunks = BN / 32;
            const int c0 = half * (BN / 2);
            uint32_t r[kChunks][16];
#pragma unroll
            for (int q = 0; q < kChunks; ++q)
                if (n0 + c0 + 16 * q < N) tmem_ld16_nowait(trow + (uint32_t)(c0 + 16 * q), r[q]);
            tmem_wait_ld();
            // the accumulator can go back to the MMA issuer before the functor runs
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty(acc));
#pragma unroll
            for (int q = 0; q < kChunks; ++q) {
                if (n0 + c0 + 16 * q >= N) break;    // warp-uniform
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[q][i]);
                if (row < M) {
                    if constexpr (BATCHED) epi(z, row, n0 + c0 + 16 * q, v);
                    else epi(row, n0 + c0 + 16 * q, v);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 2 * BN);
}

// Launches gemm_kernel over all tiles of `batch` products, one persistent CTA per SM (at most
// one per tile).  The function attribute (dynamic shared memory) is set unless the stream is
// capturing a graph (the callers set it once beforehand).
template <int BN, int STAGES, class Epi, bool BATCHED = false>
cudaError_t gemm_launch(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, int batch,
                        const Epi& epi, int* err, cudaStream_t st) {
    auto kern = gemm_kernel<BN, STAGES, Epi, BATCHED>;
    const int smem = Layout<BN, STAGES>::kBytes;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusNone) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)((M + BM - 1) / BM) * ((N + BN - 1) / BN) * batch;
    const long long grid = tiles < sms ? tiles : sms;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kGemmThreads, smem, st>>>(ta, tb, M, N, K, batch, epi, err);
    return cudaGetLastError();
}

}  // namespace tc

// ---- host side: tensor maps ---------------------------------------------------------------
// A 2-D BF16 tensor map over a row-major [rows][cols] matrix with row stride ld (elements),
// box = 64 columns x box_rows rows, 128-byte swizzle, zero fill outside the matrix.
// Returns cudaErrorInvalidValue for shapes TMA cannot describe (ld * 2 not a multiple of 16).
cudaError_t rs_make_tmap_bf16(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld,
                              int box_rows);
// Rank-3 variant over [batch][rows][cols] (row stride ld, batch stride rows * ld elements):
// box = 64 columns x box_rows rows x 1 batch; rows beyond `rows` read as zero.
cudaError_t rs_make_tmap_bf16_3d(CUtensorMap* map, const void* ptr, int64_t batch, int64_t rows, int64_t cols,
                                 int64_t ld, int box_rows);
// A [rows][K] BF16 operand (row stride ld) seen as `slices` consecutive K ranges of K / slices
// columns: a rank-3 map (K / slices, rows, slices) whose third coordinate selects the range
// (split-K with the batched GEMM kernel).  K / slices * 2 bytes must be a multiple of 16.
cudaError_t rs_make_tmap_bf16_kslices(CUtensorMap* map, const void* ptr, int64_t rows, int64_t K, int64_t ld,
                                      int slices, int box_rows);
