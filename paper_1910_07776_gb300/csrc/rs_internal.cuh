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

// Dynamic shared memory that caps a kernel at maxb resident blocks per SM (0: no cap): with
// fewer blocks than the SMs can hold at once, the block scheduler may stack them on some SMs
// and leave others idle; a cap spreads them.  static_bytes: the kernel's own shared memory.
inline size_t rs_residency_pad(int maxb, size_t static_bytes) {
    if (maxb <= 0) return 0;
    const size_t per = (size_t)228 * 1024 / (size_t)maxb;        // shared memory per SM / cap
    const size_t own = static_bytes + 1024;                      // + the block's reserved 1 KB
    return per > own ? per - own : 0;
}

// Host-side argument rules shared by every entry point that takes a batch or a set of splits:
// nullptr when the arguments are acceptable, else the reason.
inline const char* rs_batch_problem(const rs_batch* b, bool need_raw) {
    if (!b) return "batch is NULL";
    if (b->n_programs < 1) return "n_programs must be >= 1";
    if (b->max_versions < 1 || b->max_versions > RS_MAXV) return "max_versions must be in 1..64";
    if (b->max_feat < 1 || b->max_feat > 4096) return "max_feat must be in 1..4096";
    if (b->x_elems < 0) return "x_elems must be >= 0";
    if (!b->row_offsets || !b->feat_width || !b->x_offsets || !b->X || !b->masks || !b->log_time)
        return "a required batch pointer is NULL";
    if (need_raw && b->dtype != RS_F32 && b->dtype != RS_F64) return "dtype must be RS_F32 or RS_F64";
    if ((uintptr_t)b->X % (b->dtype == RS_F32 ? 4 : 8) != 0) return "X is misaligned";
    return nullptr;
}
inline const char* rs_splits_problem(const rs_splits* s) {
    if (!s) return "splits is NULL";
    if (s->n_splits < 0) return "n_splits must be >= 0";
    if (s->n_splits > 0 && (!s->split_offsets || !s->train_masks)) return "a required splits pointer is NULL";
    if (s->n_splits > (int64_t)4096 * 4096) return "at most 16,777,216 splits per call";
    if (s->max_train < 0 || s->max_train > RS_MAXV) return "max_train must be in 0..64";
    if (s->n_test_rows < 0 || s->n_test_rows > s->n_splits * (int64_t)RS_MAXV)
        return "n_test_rows must be in 0..64 * n_splits";
    return nullptr;
}

__device__ __forceinline__ uint64_t rs_full_mask(int V) {
    return V >= 64 ? ~0ull : ((1ull << V) - 1ull);
}

// Transfer (Table 2): the training runs of problem q are runs group_off[q] .. group_off[q+1]-1,
// concatenated into one list of N versions (run r's versions at start[r] .. start[r+1]-1).
// Checks 1..max_runs runs (inside the n_runs runs of the training set) of 1..64 versions, each of width F == fw_test[q] (the width of the
// problem's test program) with 1 <= F <= stat_stride.  Returns N, or -1 if a check fails.
__device__ __forceinline__ int rs_group_layout(int q, const int64_t* group_off, int max_runs, int64_t n_runs,
                                               const int64_t* row_off, const int32_t* fw, const int32_t* fw_test,
                                               int stat_stride, int (&start)[RS_MAXRUNS + 1], int& F) {
    const int64_t g0 = group_off[q], g1 = group_off[q + 1];
    if (g0 < 0 || g1 > n_runs || g1 - g0 < 1 || g1 - g0 > max_runs || g1 - g0 > RS_MAXRUNS) return -1;
    const int R = (int)(g1 - g0);
    F = fw_test[q];
    if (F < 1 || F > stat_stride) return -1;
    int N = 0;
    for (int r = 0; r < RS_MAXRUNS + 1; ++r) start[r] = 0;
    for (int r = 0; r < R; ++r) {
        const int64_t V = row_off[g0 + r + 1] - row_off[g0 + r];
        if (V < 1 || V > RS_MAXV || fw[g0 + r] != F) return -1;
        N += (int)V;
        start[r + 1] = N;
    }
    for (int r = R + 1; r < RS_MAXRUNS + 1; ++r) start[r] = N;
    return N;
}

// ---- launchers (defined in the kernel translation units) -------------------------------
cudaError_t rs_launch_standardize(const rs_batch* b, double* Z, double* mu, double* sigma,
                                  int* dstatus, cudaStream_t st);
cudaError_t rs_launch_gram_f64(const rs_batch* b, double* K, int* dstatus, cudaStream_t st);
cudaError_t rs_launch_dist2_f64(const rs_batch* b, double* K, int* dstatus, cudaStream_t st);
cudaError_t rs_launch_transfer_standardize(const rs_batch* train, const rs_batch* test, const int64_t* group_off,
                                           int max_runs, int stat_stride, double* ZA, double* ZB, double* mu,
                                           double* sigma, int* dstatus, cudaStream_t st);
// Blocks of a transfer: KA[q] (ld x ld, the group's Gram, ridge only) and Kx[q] (64 x ld:
// test row t against group version u, dot products or, with dist, squared distances).
cudaError_t rs_launch_transfer_blocks(const rs_batch* train_std, const rs_batch* test_std, const int64_t* group_off,
                                      int max_runs, int stat_stride, int ld, double* KA, double* Kx, int dist,
                                      cudaStream_t st);
size_t rs_gram_tc_workspace_bytes(int64_t P, int max_feat);
// tile_n: 32 or 64 output columns per tile; ksplit: 1 or 3 (see k_gram_tc.cu).
cudaError_t rs_launch_gram_bf16x3_ws(const rs_batch* b, double* K, void* ws, size_t ws_bytes, int* dstatus,
                                     cudaStream_t st, int tile_n = 64, int ksplit = 1);
cudaError_t rs_launch_rec_offsets(const rs_batch* b, const rs_splits* s, int64_t* rec_offsets,
                                  int64_t* scratch_blocksums, int* dstatus, cudaStream_t st);
size_t rs_rec_offsets_scratch_elems(int64_t n_splits);

// The surrogate's plain fallback (k_fallback.cu): scratch carved from the caller's workspace.
struct rs_fallback_ws {
    long long* totals;        // [8]: programs, rows, X elements, splits, test rows, features, merged rows
    int32_t* prog_map;        // [P] sub-batch index of each program, -1 if not selected
    int32_t* sub_prog;        // [P] program of each sub-batch entry
    int64_t* sub_row_off;     // [P+1]
    int64_t* sub_x_off;       // [P]
    int64_t* sub_feat_off;    // [P+1]
    int64_t* sub_split_off;   // [P+1]
    int32_t* sub_fw;          // [P]
    void* sX;                 // the selected programs' X
    uint8_t* s_masks;
    double* s_lt;
    double* s_cyc;
    uint64_t* s_train;
    int64_t* s_rec_off;       // [S+1]
    uint32_t* s_code;         // [rows cap]
    double* s_pred;           // [rows cap][k]
    void* cv_ws;              // rs_cv_step's workspace for the sub-batch
    size_t cv_ws_bytes;
    size_t bytes;             // total
};
// Pooled ridge fits in primal form (k_pooled.cu).
size_t rs_pooled_workspace_bytes_impl(int64_t P, int F);
cudaError_t rs_launch_fit_pooled(const rs_batch* b, const uint8_t* use, double lambda, int refine, void* ws,
                                 size_t ws_bytes, double* coef, uint8_t* status, int* dstatus, cudaStream_t st);
cudaError_t rs_launch_predict_pooled(const rs_batch* b, const double* coef, const uint8_t* status, int k,
                                     double log_tau, int flags, uint32_t* rec_code, double* rec_pred,
                                     double* pred_all, unsigned long long* counters, int* dstatus, cudaStream_t st);
cudaError_t rs_launch_fallback_select(const rs_batch* b, const rs_splits* sp, const uint8_t* used,
                                      const rs_fallback_ws& w, cudaStream_t st);
cudaError_t rs_launch_fallback_gather(const rs_batch* b, const rs_splits* sp, int Q, const rs_fallback_ws& w,
                                      cudaStream_t st);
cudaError_t rs_launch_fallback_merge(const rs_batch* b, const uint8_t* used, const rs_fallback_ws& w, int k,
                                     uint32_t* rec_code, double* rec_pred, cudaStream_t st);

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
    int tune_order;               // register solvers' work order: 0 largest fits first, 1 from both ends
    int64_t rows_cap;             // rows of the prediction buffer (>= rec_offsets[S])
    void* workspace;
    size_t workspace_bytes;
    // optional stage events (recorded on the stream before and after each internal launch)
    cudaEvent_t* ev;
    // optional second stream and fork/join events: the solver of the largest fits runs on
    // `side` beside the others (all three NULL: everything on the call's stream)
    cudaStream_t side;
    cudaEvent_t fork, join;
    // batched form: 0 the whole call; 1 only the planning (pairs, plan, bucket: no K read);
    // 2 only what follows it (K's diagonal, solvers, rank pass), after a phase-1 call with
    // the same arguments and workspace
    int phase;
};
#define RS_NSTAGE_EVENTS 7   // before pairs, after pairs / plan / bucket / solve / solve-large / rank
size_t rs_fit_workspace_bytes_impl(int64_t P, int64_t S, int max_train, int64_t rows_cap);
cudaError_t rs_launch_fit_predict(const rs_fit_args& a, cudaStream_t st);
// Table 2 transfer: fits of each problem's training group, predictions for its test program,
// ranking and scoring (one block per problem).
struct rs_transfer_args {
    int Q;
    const int64_t* group_off;     // [Q+1]
    int max_runs;
    int64_t n_runs;               // runs of the training set
    int stat_stride;
    const int64_t* a_row_offsets;
    const int32_t* a_feat_width;
    const uint8_t* a_masks;
    const double* a_log_time;
    const int64_t* b_row_offsets;
    const int32_t* b_feat_width;
    const uint8_t* b_masks;
    const double* b_log_time;
    const double* KA;             // [Q][ld][ld] group Gram (ridge)
    const double* Kx;             // [Q][64][ld] cross block (dot products, or squared distances for IBK)
    int ld;
    double lambda;
    int ibk;
    int opt_mask;
    int k;
    double log_tau;
    int flags;
    uint8_t* fit_status;          // [Q][6], nullable
    double* fit_ws;               // rs_transfer_fit_bytes(Q) of device scratch for the ridge fits
    int m5p;                      // the M5P model tree (RS_MODEL_M5P)
    void* m5_ws;                  // Q * 6 * rs_m5p_tree_bytes() of device scratch for its trees
    const double* ZA;             // standardized training rows (train's x_offsets)
    const int64_t* a_x_offsets;
    const double* ZB;             // standardized test rows (test's x_offsets)
    const int64_t* b_x_offsets;
    uint32_t* rec_code;
    double* rec_pred;
    double* pred_all;
    unsigned long long* counters;
    int* dstatus;
};
cudaError_t rs_launch_transfer(const rs_transfer_args& a, cudaStream_t st);
size_t rs_transfer_fit_bytes(int64_t Q);
size_t rs_m5p_tree_bytes();
int rs_m5p_max_feat();
cudaError_t rs_launch_iota64(int64_t* out, int64_t n, cudaStream_t st);
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
