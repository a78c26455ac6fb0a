// tc_gemm.cuh -- BF16 GEMM on the sm_103a tensor cores (tcgen05), used by the surrogate's
// forward / backward kernels and by the tensor-core Gram.
//
//   D[M][N] (FP32, in tensor memory) = A[M][K] * B[N][K]^T,  A, B BF16, both K-contiguous.
//
// One CTA (4 warps) owns a 128 x BN tile of D.  Thread 0 drives a STAGES-deep ring of shared
// memory stages: TMA 2-D loads (128-byte swizzle) of a 128 x 64 slice of A and a BN x 64
// slice of B complete on the stage's "full" mbarrier; four tcgen05.mma (M=128, N=BN, K=16)
// per stage accumulate into tensor memory; tcgen05.commit on the stage's "empty" mbarrier
// frees the stage for the next TMA.  After the last k-block a commit on "done" releases the
// epilogue: each warp reads its 32 accumulator rows with tcgen05.ld (16 columns at a time)
// and hands them to the epilogue functor.  Every mbarrier wait is bounded (1 s of
// %globaltimer); a wait that gives up sets RS_ETIMEOUT in the device status word, the CTA
// skips the epilogue, frees its tensor memory and returns.
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

// Epi: __device__ void operator()(int row, int col0, const float (&v)[16]) const; called for
// every row < M of the tile with the 16 accumulator columns starting at col0 (col0 < N).
// BATCHED: the operands are rank-3 tensor maps [batch][rows][K]; CTA z works on batch z and
// the epilogue is called as epi(z, row, col0, v).
template <int BN, int STAGES, class Epi, bool BATCHED = false>
__global__ void __launch_bounds__(128, 1)
gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, int M, int N,
            int K, Epi epi, int* err) {
    using L = Layout<BN, STAGES>;
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256 && (BN & (BN - 1)) == 0, "BN: 32..256, power of 2");
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gbase = smem_raw + (base - raw);
    const uint32_t bars = base + STAGES * L::kStage;            // full[S], empty[S], done
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gbase + STAGES * L::kStage + 8 * (2 * STAGES + 1));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int nk = (K + BK - 1) / BK;
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (STAGES + s); };
    const uint32_t done = bars + 8u * (2 * STAGES);

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(done, 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(tmem_slot), BN);
        tmem_relinquish();
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (tid == 0) {
        const uint32_t idesc = idesc_bf16(BM, BN);
        const int pre = nk < STAGES ? nk : STAGES;
        int issued = 0, consumed = 0;
        auto load = [&](int kb, uint32_t a, uint32_t b, uint32_t bar) {
            mbar_expect_tx(bar, L::kStage);
            if (BATCHED) {
                tma_load_3d(a, &ta, bar, kb * BK, m0, blockIdx.z);
                tma_load_3d(b, &tb, bar, kb * BK, n0, blockIdx.z);
            } else {
                tma_load_2d(a, &ta, bar, kb * BK, m0);
                tma_load_2d(b, &tb, bar, kb * BK, n0);
            }
        };
        for (int kb = 0; kb < pre; ++kb, ++issued) {
            const uint32_t a = base + kb * L::kStage, b = a + L::kA;
            load(kb, a, b, full(kb));
        }
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % STAGES;
            ok = mbar_wait(full(s), (kb / STAGES) & 1, err, 1);
            if (!ok) break;
            ++consumed;
            fence_after();
            const uint32_t a = base + s * L::kStage, b = a + L::kA;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem, sw128_desc(a + kk * 32), sw128_desc(b + kk * 32), idesc, (kb | kk) != 0);
            mma_commit(empty(s));
            // refill the stage used one iteration ago (its MMAs are queued behind these)
            const int kr = kb - 1 + STAGES;
            if (kb >= 1 && kr < nk) {
                const int sp = (kb - 1) % STAGES;
                ok = mbar_wait(empty(sp), ((kb - 1) / STAGES) & 1, err, 2);
                if (!ok) break;
                const uint32_t a2 = base + sp * L::kStage, b2 = a2 + L::kA;
                load(kr, a2, b2, full(sp));
                ++issued;
            }
        }
        if (!ok)   // a wait gave up: wait (bounded) for the loads still in flight before leaving
            for (int kb = consumed; kb < issued; ++kb) mbar_wait(full(kb % STAGES), (kb / STAGES) & 1, err, 4);
        mma_commit(done);
    }
    __syncwarp();
    ok = mbar_wait(done, 0, err, 3);
    fence_after();
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
            if (n0 + c >= N) break;                  // warp-uniform
            float v[16];
            tmem_ld16(trow + (uint32_t)c, v);
            if (row < M) {
                if constexpr (BATCHED) epi((int)blockIdx.z, row, n0 + c, v);
                else epi(row, n0 + c, v);
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, BN);
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
