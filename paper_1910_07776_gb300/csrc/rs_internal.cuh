// rs_internal.cuh -- declarations shared by the library's translation units (device side
// and host launchers).  Nothing here is visible through the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rs.h"

// Device status word layout (ints in the context's 4 KiB device area).
#define RS_DST_CODE 0      // first error code seen by a kernel (rs_status values)
#define RS_DST_DETAIL 1    // a detail (program index, wait site) for that error
#define RS_DST_QUEUE 16    // unsigned queue heads for persistent kernels (8 slots)
#define RS_DST_INTS 1024

struct rs_ctx_dev {
    int* status;           // [RS_DST_INTS] in device memory
};

__device__ __forceinline__ void rs_dev_flag(int* status, int code, int detail) {
    if (status == nullptr) return;
    if (atomicCAS(status + RS_DST_CODE, 0, code) == 0) status[RS_DST_DETAIL] = detail;
}

// Binary search: the program p with offs[p] <= i < offs[p+1] (offs has P+1 entries).
__device__ __forceinline__ int rs_find_segment(const int64_t* offs, int P, int64_t i) {
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint64_t rs_full_mask(int V) {
    return V >= 64 ? ~0ull : ((1ull << V) - 1ull);
}

// ---- launchers (defined in the kernel translation units) -------------------------------
cudaError_t rs_launch_standardize(const rs_batch* b, double* Z, double* mu, double* sigma,
                                  int* dstatus, cudaStream_t st);
cudaError_t rs_launch_gram_f64(const rs_batch* b, double* K, int* dstatus, cudaStream_t st);
cudaError_t rs_launch_dist2_f64(const rs_batch* b, double* K, int* dstatus, cudaStream_t st);
size_t rs_gram_tc_workspace_bytes(int64_t P, int max_feat);
cudaError_t rs_launch_gram_bf16x3_ws(const rs_batch* b, double* K, void* ws, size_t ws_bytes, int* dstatus,
                                     cudaStream_t st);
cudaError_t rs_launch_rec_offsets(const rs_batch* b, const rs_splits* s, int64_t* rec_offsets,
                                  int64_t* scratch_blocksums, int* dstatus, cudaStream_t st);
size_t rs_rec_offsets_scratch_elems(int64_t n_splits);

struct rs_fit_args {
    // batch (standardized)
    int P;
    const int64_t* row_offsets;
    const int32_t* feat_width;
    const int64_t* x_offsets;
    const double* Z;
    const uint8_t* masks;
    const double* log_time;
    const double* K;
    // splits
    int64_t S;
    const int64_t* split_offsets;
    const uint64_t* train_masks;
    // parameters
    double lambda;
    int k;
    double log_tau;
    int flags;
    int form;
    // inputs/outputs (nullable unless noted)
    const double* coef_in;
    double* coef_out;
    uint8_t* status_out;
    const int64_t* rec_offsets;   // required for ranking
    uint32_t* rec_code;           // if NULL: fit only
    double* rec_pred;
    double* pred_all;
    unsigned long long* counters;
    int* dstatus;
    unsigned int* queue;          // persistent work queue head (zeroed before launch)
    // batched form only
    int max_train;                // host bound on popcount(train mask)
    int max_feat;                 // host bound on F_p (refinement buffers)
    int tune_split;               // largest n of the lighter one-fit-per-thread solver (4..8)
    int tune_rank_waves;          // rank-pass grid = SMs x this (0: default)
    int64_t rows_cap;             // rows of the prediction buffer (>= rec_offsets[S])
    void* workspace;
    size_t workspace_bytes;
    // optional stage events (recorded on the stream before and after each internal launch)
    cudaEvent_t* ev;
    // optional second stream and fork/join events: the solver of the largest fits runs on
    // `side` beside the others (all three NULL: everything on the call's stream)
    cudaStream_t side;
    cudaEvent_t fork, join;
};
#define RS_NSTAGE_EVENTS 7   // before pairs, after pairs / plan / bucket / solve / solve-large / rank
size_t rs_fit_workspace_bytes_impl(int64_t P, int64_t S, int max_train, int64_t rows_cap);
cudaError_t rs_launch_fit_predict(const rs_fit_args& a, cudaStream_t st);
size_t rs_surrogate_blob_floats();
size_t rs_surrogate_train_ws_bytes(int B);
size_t rs_surrogate_infer_ws_bytes(int64_t chunk);
int64_t rs_surrogate_blob_offset(int which);
cudaError_t rs_launch_surrogate_train(float* blob, const double* X, const double* Y, int64_t n, int B,
                                      int64_t steps, float lr, float wd, float* loss_curve, void* ws,
                                      int use_graph, int* err, cudaStream_t st);
cudaError_t rs_launch_surrogate_infer(const float* blob, const double* X, int64_t n, float ood_thr,
                                      float* pred, float* score, uint8_t* fallback, const uint8_t* masks,
                                      int k, double tau, int flags, uint32_t* rec_code, double* rec_pred,
                                      void* ws, int64_t chunk, int* err, cudaStream_t st);
cudaError_t rs_launch_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, float* D, int64_t ldd,
                                int M, int N, int K, int* err, cudaStream_t st);
