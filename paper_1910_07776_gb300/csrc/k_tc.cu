// Tensor maps for the tcgen05 GEMM core, and rs_gemm_bf16: a plain BF16 GEMM with FP32
// output on the tensor cores (the building block of the surrogate and the tensor-core Gram).
#include "tc_gemm.cuh"

#include <cudaTypedefs.h>

#include <mutex>

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

void load_encode() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
}

struct EpiStoreF32 {
    float* D;
    int64_t ldd;
    int N;
    __device__ void operator()(int row, int col0, const float (&v)[16]) const {
        float* d = D + (int64_t)row * ldd + col0;
        if (col0 + 16 <= N && ((uintptr_t)d & 15) == 0) {   // whole aligned chunk: 16-byte stores
            float4* d4 = reinterpret_cast<float4*>(d);
#pragma unroll
            for (int q = 0; q < 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            return;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (col0 + i < N) d[i] = v[i];
    }
};

}  // namespace

cudaError_t rs_make_tmap_bf16(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld,
                              int box_rows) {
    std::call_once(g_encode_once, load_encode);
    if (!g_encode) return cudaErrorNotSupported;
    if (rows < 1 || cols < 1 || ld < cols || (ld * 2) % 16 != 0 || ((uintptr_t)ptr % 16) != 0)
        return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t rs_make_tmap_bf16_3d(CUtensorMap* map, const void* ptr, int64_t batch, int64_t rows, int64_t cols,
                                 int64_t ld, int box_rows) {
    std::call_once(g_encode_once, load_encode);
    if (!g_encode) return cudaErrorNotSupported;
    if (batch < 1 || rows < 1 || cols < 1 || ld < cols || (ld * 2) % 16 != 0 || ((uintptr_t)ptr % 16) != 0)
        return cudaErrorInvalidValue;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(rows * ld * 2)};
    cuuint32_t box[3] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t rs_make_tmap_bf16_kslices(CUtensorMap* map, const void* ptr, int64_t rows, int64_t K, int64_t ld,
                                      int slices, int box_rows) {
    std::call_once(g_encode_once, load_encode);
    if (!g_encode) return cudaErrorNotSupported;
    if (slices < 1 || rows < 1 || K < slices || K % slices || ld < K || (ld * 2) % 16 != 0 ||
        ((K / slices) * 2) % 16 != 0 || ((uintptr_t)ptr % 16) != 0)
        return cudaErrorInvalidValue;
    const int64_t ks = K / slices;
    cuuint64_t dims[3] = {(cuuint64_t)ks, (cuuint64_t)rows, (cuuint64_t)slices};
    cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(ks * 2)};
    cuuint32_t box[3] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(ptr), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN>
static cudaError_t launch_store(const CUtensorMap& ta, const CUtensorMap& tb, int M, int N, int K, float* D,
                                int64_t ldd, int* err, cudaStream_t st) {
    return tc::gemm_launch<BN, 4, EpiStoreF32>(ta, tb, M, N, K, 1, EpiStoreF32{D, ldd, N}, err, st);
}

cudaError_t rs_launch_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* D, int64_t ldd,
                                int M, int N, int K, int* err, cudaStream_t st) {
    CUtensorMap ta, tb;
    const int bn = N > 128 ? 256 : 128;
    cudaError_t e = rs_make_tmap_bf16(&ta, A, M, K, lda, tc::BM);
    if (e == cudaSuccess) e = rs_make_tmap_bf16(&tb, B, N, K, ldb, bn);
    if (e != cudaSuccess) return e;
    return bn == 256 ? launch_store<256>(ta, tb, M, N, K, D, ldd, err, st)
                     : launch_store<128>(ta, tb, M, N, K, D, ldd, err, st);
}
