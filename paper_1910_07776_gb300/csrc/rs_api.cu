// rs_api.cu -- host side of the C ABI declared in include/rs.h: argument validation,
// context state, and the launch sequence of each entry point.  No arithmetic of the
// method happens here; every step runs in the kernels of the k_*.cu files.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "rs_internal.cuh"

struct rs_ctx {
    int device;
    cudaStream_t stream;
    int* dstatus;            // RS_DST_INTS ints of device memory
    int64_t* scan;           // block sums of the row-planning scan (kScanBlocksMax + 1)
    int profiling;           // record stage events in the batched fit/predict path
    int tune_split;          // autotuned launch parameters of the batched form
    int tune_rank_waves;
    int tune_order;
    uint8_t gram_cfg[65];    // tensor-core Gram tiles per padded width / 64: bit 0 = 32-column
                             // tiles (else 64), bit 1 = K split in three (else whole)
    cudaEvent_t ev[RS_NSTAGE_EVENTS];
    cudaStream_t side;       // second stream of the batched solver (fork/join on events)
    cudaEvent_t fork, join;
    char err[512];
};

namespace {

rs_status fail(rs_ctx* c, rs_status code, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

rs_status cuda_fail(rs_ctx* c, cudaError_t e, const char* where) {
    return fail(c, RS_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

rs_status check_batch(rs_ctx* c, const rs_batch* b, bool need_raw) {
    const char* why = rs_batch_problem(b, need_raw);
    return why ? fail(c, RS_EINVAL, "%s", why) : RS_OK;
}

rs_status check_splits(rs_ctx* c, const rs_splits* s) {
    const char* why = rs_splits_problem(s);
    return why ? fail(c, RS_EINVAL, "%s", why) : RS_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// The tensor-core Gram's tuning slot of a feature width: its width rounded up to 64, / 64.
int gram_slot(int max_feat) {
    const int s = (max_feat + 63) / 64;
    return s < 1 ? 1 : (s > 64 ? 64 : s);
}

}  // namespace

extern "C" {

rs_status rs_create(rs_ctx** out, int device, void* stream) {
    if (!out) return RS_EINVAL;
    *out = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return RS_ECUDA;
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return RS_ECUDA;
    if (!(prop.major == 10 && prop.minor == 3)) return RS_EUNSUPPORTED;
    rs_ctx* c = new (std::nothrow) rs_ctx;
    if (!c) return RS_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    c->err[0] = 0;
    c->profiling = 0;
    c->tune_split = 6;
    c->tune_rank_waves = 32;
    c->tune_order = 1;      // measured: the solver group 7 % faster than largest-first on the
                            // batched-CV workload (0.430 vs 0.462 ms)
    memset(c->gram_cfg, 0, sizeof(c->gram_cfg));   // 64-column tiles, whole K
    for (int i = 0; i < RS_NSTAGE_EVENTS; ++i) c->ev[i] = nullptr;
    c->side = nullptr;
    c->fork = c->join = nullptr;
    e = cudaMalloc(&c->dstatus, RS_DST_INTS * sizeof(int));
    if (e != cudaSuccess) {
        delete c;
        return RS_ECUDA;
    }
    e = cudaMalloc(&c->scan, rs_rec_offsets_scratch_elems((int64_t)4096 * 4096) * sizeof(int64_t));
    if (e != cudaSuccess) {
        cudaFree(c->dstatus);
        delete c;
        return RS_ECUDA;
    }
    e = cudaMemset(c->dstatus, 0, RS_DST_INTS * sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(c->dstatus);
        cudaFree(c->scan);
        delete c;
        return RS_ECUDA;
    }
    // the side stream is an optimisation: without it every launch stays on the call's stream
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->side) cudaStreamDestroy(c->side);
        if (c->fork) cudaEventDestroy(c->fork);
        if (c->join) cudaEventDestroy(c->join);
        c->side = nullptr;
        c->fork = c->join = nullptr;
    }
    *out = c;
    return RS_OK;
}

rs_status rs_destroy(rs_ctx* c) {
    if (!c) return RS_EINVAL;
    cudaSetDevice(c->device);
    cudaFree(c->dstatus);
    cudaFree(c->scan);
    for (int i = 0; i < RS_NSTAGE_EVENTS; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->join) cudaEventDestroy(c->join);
    delete c;
    return RS_OK;
}

rs_status rs_profile_enable(rs_ctx* c, int on) {
    if (!c) return RS_EINVAL;
    cudaSetDevice(c->device);
    if (on && !c->ev[0])
        for (int i = 0; i < RS_NSTAGE_EVENTS; ++i) {
            cudaError_t e = cudaEventCreate(&c->ev[i]);
            if (e != cudaSuccess) return cuda_fail(c, e, "rs_profile_enable");
        }
    c->profiling = on ? 1 : 0;
    return RS_OK;
}

rs_status rs_profile_read(rs_ctx* c, float* ms, int max_stages, int* n_stages) {
    if (!c || !ms || !n_stages) return RS_EINVAL;
    *n_stages = 0;
    if (!c->profiling) return fail(c, RS_EINVAL, "profiling is off");
    cudaSetDevice(c->device);
    cudaError_t e = cudaEventSynchronize(c->ev[RS_NSTAGE_EVENTS - 1]);
    if (e != cudaSuccess) return cuda_fail(c, e, "rs_profile_read");
    int n = 0;
    for (int i = 0; i + 1 < RS_NSTAGE_EVENTS && n < max_stages; ++i, ++n) {
        e = cudaEventElapsedTime(&ms[n], c->ev[i], c->ev[i + 1]);
        if (e != cudaSuccess) return cuda_fail(c, e, "rs_profile_read");
    }
    *n_stages = n;
    return RS_OK;
}

rs_status rs_set_stream(rs_ctx* c, void* stream) {
    if (!c) return RS_EINVAL;
    c->stream = (cudaStream_t)stream;
    return RS_OK;
}

const char* rs_last_error(const rs_ctx* c) { return c ? c->err : "context is NULL"; }

rs_status rs_check_device_status(rs_ctx* c) {
    if (!c) return RS_EINVAL;
    cudaSetDevice(c->device);
    int h[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(h, c->dstatus, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "rs_check_device_status");
    if (h[0] != 0) {
        e = cudaMemsetAsync(c->dstatus, 0, 2 * sizeof(int), c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "rs_check_device_status");
        if (h[0] == RS_EDATA) return fail(c, RS_EDATA, "program %d has fewer than 1 or more than 64 versions", h[1]);
        if (h[0] == RS_ETIMEOUT) return fail(c, RS_ETIMEOUT, "a bounded device wait gave up (site %d)", h[1]);
        return fail(c, (rs_status)h[0], "device status %d (detail %d)", h[0], h[1]);
    }
    return RS_OK;
}

rs_status rs_standardize(rs_ctx* c, const rs_batch* b, double* Z, double* mu, double* sigma) {
    if (!c) return RS_EINVAL;
    rs_status s = check_batch(c, b, true);
    if (s != RS_OK) return s;
    if (!Z) return fail(c, RS_EINVAL, "Z is NULL");
    if ((mu || sigma) && !b->feat_offsets) return fail(c, RS_EINVAL, "feat_offsets is NULL");
    cudaSetDevice(c->device);
    cudaError_t e = rs_launch_standardize(b, Z, mu, sigma, c->dstatus, c->stream);
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_standardize");
}

size_t rs_gram_workspace_bytes(const rs_batch* b, int precision) {
    if (!b || b->n_programs < 1 || b->max_feat < 1) return 0;
    return precision == RS_GRAM_BF16X3 ? rs_gram_tc_workspace_bytes(b->n_programs, b->max_feat) : 0;
}

rs_status rs_gram(rs_ctx* c, const rs_batch* b, int precision, double* K, void* ws, size_t ws_bytes) {
    if (!c) return RS_EINVAL;
    rs_status s = check_batch(c, b, false);
    if (s != RS_OK) return s;
    if (!K) return fail(c, RS_EINVAL, "K is NULL");
    cudaSetDevice(c->device);
    cudaError_t e;
    if (precision == RS_GRAM_F64) {
        e = rs_launch_gram_f64(b, K, c->dstatus, c->stream);
    } else if (precision == RS_GRAM_DIST2) {
        e = rs_launch_dist2_f64(b, K, c->dstatus, c->stream);
    } else if (precision == RS_GRAM_BF16X3) {
        const size_t need = rs_gram_workspace_bytes(b, precision);
        if (!ws || ws_bytes < need) return fail(c, RS_ENOMEM, "the tensor-core Gram needs %zu bytes of workspace", need);
        if ((uintptr_t)ws % 256) return fail(c, RS_EINVAL, "workspace must be 256-byte aligned");
        if (b->n_programs > 65535) return fail(c, RS_EINVAL, "the tensor-core Gram takes at most 65535 programs per call");
        const int cfg = c->gram_cfg[gram_slot(b->max_feat)];
        e = rs_launch_gram_bf16x3_ws(b, K, ws, ws_bytes, c->dstatus, c->stream, (cfg & 1) ? 32 : 64,
                                     (cfg & 2) ? 3 : 1);
    } else {
        return fail(c, RS_EINVAL, "precision must be RS_GRAM_F64, RS_GRAM_BF16X3 or RS_GRAM_DIST2");
    }
    if (e == cudaErrorNotSupported) return fail(c, RS_EUNSUPPORTED, "rs_gram: cuTensorMapEncodeTiled unavailable");
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_gram");
}

}  // extern "C"

extern "C" {

rs_status rs_rec_offsets(rs_ctx* c, const rs_batch* b, const rs_splits* sp, int64_t* ro) {
    if (!c) return RS_EINVAL;
    rs_status s = check_batch(c, b, false);
    if (s == RS_OK) s = check_splits(c, sp);
    if (s != RS_OK) return s;
    if (!ro) return fail(c, RS_EINVAL, "rec_offsets is NULL");
    cudaSetDevice(c->device);
    cudaError_t e = rs_launch_rec_offsets(b, sp, ro, c->scan, c->dstatus, c->stream);
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_rec_offsets");
}

static rs_status fit_common(rs_ctx* c, const rs_batch* b, const double* K, const rs_splits* sp,
                            double lambda, int form, rs_fit_args& a) {
    rs_status s = check_batch(c, b, false);
    if (s == RS_OK) s = check_splits(c, sp);
    if (s != RS_OK) return s;
    if (!K) return fail(c, RS_EINVAL, "K is NULL");
    if (!(lambda >= 0.0) || !isfinite(lambda)) return fail(c, RS_EINVAL, "lambda must be finite and >= 0");
    if (form != RS_FORM_BATCHED && form != RS_FORM_PLAIN) return fail(c, RS_EINVAL, "bad form");
    memset(&a, 0, sizeof(a));
    a.P = b->n_programs;
    a.row_offsets = b->row_offsets;
    a.feat_width = b->feat_width;
    a.x_offsets = b->x_offsets;
    a.Z = (const double*)b->X;
    a.masks = b->masks;
    a.log_time = b->log_time;
    a.K = K;
    a.S = sp->n_splits;
    a.split_offsets = sp->split_offsets;
    a.train_masks = sp->train_masks;
    a.lambda = lambda;
    a.form = form;
    a.max_feat = b->max_feat;
    a.dstatus = c->dstatus;
    a.queue = (unsigned int*)(c->dstatus + RS_DST_QUEUE);
    a.ev = c->profiling ? c->ev : nullptr;
    a.tune_split = c->tune_split;
    a.tune_rank_waves = c->tune_rank_waves;
    a.tune_order = c->tune_order;
    a.side = c->side;
    a.fork = c->fork;
    a.join = c->join;
    return RS_OK;
}

static int64_t rows_cap(const rs_batch* b, const rs_splits* sp) {
    return sp->n_test_rows > 0 ? sp->n_test_rows : sp->n_splits * (int64_t)b->max_versions;
}

size_t rs_fit_workspace_bytes(const rs_batch* b, const rs_splits* sp) {
    if (!b || !sp || b->n_programs < 1 || sp->n_splits < 0) return 0;
    return rs_fit_workspace_bytes_impl(b->n_programs, sp->n_splits, sp->max_train, rows_cap(b, sp));
}

static rs_status check_ws(rs_ctx* c, const rs_batch* b, const rs_splits* sp, void* ws, size_t bytes,
                          rs_fit_args& a) {
    const size_t need = rs_fit_workspace_bytes(b, sp);
    if (!ws) return fail(c, RS_EINVAL, "the batched form needs a workspace of %zu bytes", need);
    if ((uintptr_t)ws % 256 != 0) return fail(c, RS_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < need) return fail(c, RS_ENOMEM, "workspace has %zu bytes, needs %zu", bytes, need);
    if (sp->max_train < 0 || sp->max_train > 64) return fail(c, RS_EINVAL, "max_train must be in 0..64");
    a.workspace = ws;
    a.workspace_bytes = bytes;
    a.max_train = sp->max_train;
    a.rows_cap = rows_cap(b, sp);
    return RS_OK;
}

rs_status rs_fit_batched(rs_ctx* c, const rs_batch* b, const double* K, const rs_splits* sp,
                         double lambda, int form, void* workspace, size_t workspace_bytes,
                         double* coef, uint8_t* fit_status) {
    if (!c) return RS_EINVAL;
    const int refine = form & RS_REFINE_X, loo = form & RS_LOO_CLOSED;
    form &= ~(RS_REFINE_X | RS_LOO_CLOSED);
    rs_fit_args a;
    rs_status s = fit_common(c, b, K, sp, lambda, form, a);
    if (s != RS_OK) return s;
    if (refine && form != RS_FORM_BATCHED) return fail(c, RS_EINVAL, "RS_REFINE_X needs the batched form");
    if (loo && (form != RS_FORM_BATCHED || refine))
        return fail(c, RS_EINVAL, "RS_LOO_CLOSED needs the batched form without RS_REFINE_X");
    if (refine && b->max_feat > 4096) return fail(c, RS_EINVAL, "RS_REFINE_X: max_feat <= 4096");
    if (form == RS_FORM_BATCHED) {
        s = check_ws(c, b, sp, workspace, workspace_bytes, a);
        if (s != RS_OK) return s;
    }
    a.flags |= refine | loo;
    a.coef_out = coef;
    a.status_out = fit_status;
    a.k = 1;
    a.log_tau = 0.0;
    cudaSetDevice(c->device);
    cudaError_t e = rs_launch_fit_predict(a, c->stream);
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_fit_batched");
}

// The checks and arguments of rs_predict_rank (no launch).
static rs_status predict_args(rs_ctx* c, const rs_batch* b, const double* K, const rs_splits* sp,
                              double lambda, const double* coef, int k, double tau, int flags,
                              int form, void* workspace, size_t workspace_bytes,
                              const int64_t* rec_offsets, uint32_t* rec_code, double* rec_pred,
                              double* pred_all, uint64_t* counters, rs_fit_args& a) {
    rs_status s = fit_common(c, b, K, sp, lambda, form, a);
    if (s != RS_OK) return s;
    if (form == RS_FORM_BATCHED && !coef) {
        s = check_ws(c, b, sp, workspace, workspace_bytes, a);
        if (s != RS_OK) return s;
    }
    if (k < 1 || k > RS_NOPT) return fail(c, RS_EINVAL, "k must be in 1..6");
    if (!(tau > 0.0) || !isfinite(tau)) return fail(c, RS_EINVAL, "tau must be finite and > 0");
    if (flags & ~(RS_RANK_ALL | RS_REFINE_X | RS_MODEL_IBK | RS_PACK_PRED | RS_LOO_CLOSED))
        return fail(c, RS_EINVAL, "unknown flag bits");
    if ((flags & RS_LOO_CLOSED) && (form != RS_FORM_BATCHED || coef || (flags & (RS_REFINE_X | RS_MODEL_IBK))))
        return fail(c, RS_EINVAL, "RS_LOO_CLOSED needs the batched form, coef = NULL, no RS_REFINE_X or RS_MODEL_IBK");
    if ((flags & RS_PACK_PRED) && (form != RS_FORM_BATCHED || coef))
        return fail(c, RS_EINVAL, "RS_PACK_PRED needs the batched form with the fits computed in the call (coef = NULL)");
    if ((flags & RS_MODEL_IBK) && (form != RS_FORM_BATCHED || coef || (flags & RS_REFINE_X)))
        return fail(c, RS_EINVAL, "RS_MODEL_IBK needs the batched form, coef = NULL and no RS_REFINE_X");
    if ((flags & RS_REFINE_X) && (form != RS_FORM_BATCHED || coef))
        return fail(c, RS_EINVAL, "RS_REFINE_X needs the batched form and refits in the call (coef = NULL)");
    if ((flags & RS_REFINE_X) && b->max_feat > 4096) return fail(c, RS_EINVAL, "RS_REFINE_X: max_feat <= 4096");
    if (!rec_offsets || !rec_code) return fail(c, RS_EINVAL, "rec_offsets and rec_code are required");
    a.coef_in = coef;
    a.k = k;
    a.log_tau = log(tau);   // host libm, the same call on both sides of any comparison
    a.flags = flags;
    a.rec_offsets = rec_offsets;
    a.rec_code = rec_code;
    a.rec_pred = rec_pred;
    a.pred_all = pred_all;
    a.counters = (unsigned long long*)counters;
    return RS_OK;
}

rs_status rs_predict_rank(rs_ctx* c, const rs_batch* b, const double* K, const rs_splits* sp,
                          double lambda, const double* coef, int k, double tau, int flags,
                          int form, void* workspace, size_t workspace_bytes,
                          const int64_t* rec_offsets, uint32_t* rec_code, double* rec_pred,
                          double* pred_all, uint64_t* counters) {
    if (!c) return RS_EINVAL;
    rs_fit_args a;
    rs_status s = predict_args(c, b, K, sp, lambda, coef, k, tau, flags, form, workspace, workspace_bytes,
                               rec_offsets, rec_code, rec_pred, pred_all, counters, a);
    if (s != RS_OK) return s;
    cudaSetDevice(c->device);
    cudaError_t e = rs_launch_fit_predict(a, c->stream);
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_predict_rank");
}

rs_status rs_gemm_bf16(rs_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, float* D,
                       int64_t ldd, int M, int N, int K) {
    if (!c) return RS_EINVAL;
    if (!A || !B || !D) return fail(c, RS_EINVAL, "A, B and D are required");
    if (M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldd < N)
        return fail(c, RS_EINVAL, "sizes: M, N, K >= 1, lda, ldb >= K, ldd >= N");
    if ((lda * 2) % 16 || (ldb * 2) % 16 || (uintptr_t)A % 16 || (uintptr_t)B % 16)
        return fail(c, RS_EINVAL, "A and B rows must start on 16-byte boundaries (lda, ldb multiples of 8)");
    cudaSetDevice(c->device);
    cudaError_t e = rs_launch_gemm_bf16(A, lda, B, ldb, D, ldd, M, N, K, c->dstatus, c->stream);
    if (e == cudaErrorNotSupported) return fail(c, RS_EUNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_gemm_bf16");
}

size_t rs_surrogate_blob_bytes(void) { return rs_surrogate_blob_floats() * sizeof(float); }

int64_t rs_surrogate_offset(int which) { return rs_surrogate_blob_offset(which); }

size_t rs_surrogate_workspace_bytes(int batch_rows) {
    if (batch_rows < 1) return 0;
    const size_t t = rs_surrogate_train_ws_bytes(batch_rows);
    const size_t i = rs_surrogate_infer_ws_bytes(batch_rows);
    return t > i ? t : i;
}

rs_status rs_surrogate_train(rs_ctx* c, float* blob, const double* X, const double* Y, int64_t n,
                             const rs_mlp_cfg* cfg, float* loss_curve, void* ws, size_t ws_bytes) {
    if (!c) return RS_EINVAL;
    if (!blob || !X || !Y || !cfg || !ws) return fail(c, RS_EINVAL, "blob, X, Y, cfg and workspace are required");
    if (n < 1 || cfg->batch_rows < 16 || cfg->batch_rows % 8 || cfg->batch_rows > n || cfg->steps < 0)
        return fail(c, RS_EINVAL, "need n >= batch_rows >= 16, batch_rows a multiple of 8, steps >= 0");
    if (!(cfg->lr >= 0.f) || !(cfg->weight_decay >= 0.f)) return fail(c, RS_EINVAL, "lr and weight_decay must be >= 0");
    if ((uintptr_t)blob % 256 || (uintptr_t)ws % 256) return fail(c, RS_EINVAL, "blob and workspace must be 256-byte aligned");
    if (ws_bytes < rs_surrogate_workspace_bytes(cfg->batch_rows))
        return fail(c, RS_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes,
                    rs_surrogate_workspace_bytes(cfg->batch_rows));
    cudaSetDevice(c->device);
    cudaError_t e = rs_launch_surrogate_train(blob, X, Y, n, cfg->batch_rows, cfg->steps, cfg->lr,
                                              cfg->weight_decay, loss_curve, ws, cfg->use_graph, c->dstatus,
                                              c->stream);
    if (e == cudaErrorNotSupported) return fail(c, RS_EUNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_surrogate_train");
}

rs_status rs_surrogate_infer(rs_ctx* c, const float* blob, const double* X, int64_t n, float ood_threshold,
                             float* pred, float* ood_score, uint8_t* used_fallback, const uint8_t* masks,
                             int k, double tau, int flags, uint32_t* rec_code, double* rec_pred, void* ws,
                             size_t ws_bytes, int chunk_rows) {
    if (!c) return RS_EINVAL;
    if (!blob || !X || !ws) return fail(c, RS_EINVAL, "blob, X and workspace are required");
    if (!pred && !rec_code) return fail(c, RS_EINVAL, "ask for pred and/or rec_code");
    if (rec_code && (k < 1 || k > RS_NOPT || !(tau > 0.0) || (flags & ~RS_RANK_ALL)))
        return fail(c, RS_EINVAL, "ranking: k in 1..6, tau > 0, flags RS_RANK_ALL only");
    if (n < 1 || chunk_rows < 16 || chunk_rows % 8) return fail(c, RS_EINVAL, "n >= 1, chunk_rows >= 16, multiple of 8");
    if ((uintptr_t)blob % 256 || (uintptr_t)ws % 256) return fail(c, RS_EINVAL, "blob and workspace must be 256-byte aligned");
    if ((uintptr_t)X % 16) return fail(c, RS_EINVAL, "X must be 16-byte aligned");
    if (ws_bytes < rs_surrogate_infer_ws_bytes(chunk_rows))
        return fail(c, RS_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, rs_surrogate_infer_ws_bytes(chunk_rows));
    cudaSetDevice(c->device);
    cudaError_t e = rs_launch_surrogate_infer(blob, X, n, ood_threshold, pred, ood_score, used_fallback, masks,
                                              k, tau, flags, rec_code, rec_pred, ws, chunk_rows, c->dstatus,
                                              c->stream);
    if (e == cudaErrorNotSupported) return fail(c, RS_EUNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_surrogate_infer");
}

// ---- surrogate checkpoints: a 64-byte header, then the blob as it is on the device
namespace {
struct CkptHeader {
    char magic[8];                // "RSSURR01"
    uint32_t version;             // 1
    uint32_t width[4];            // 256, 512, 512, 6
    uint32_t dtype;               // 0: FP32
    int64_t step;                 // optimizer steps taken (AdamW's t)
    uint64_t blob_bytes;
    unsigned char pad[16];
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");
constexpr char kCkptMagic[8] = {'R', 'S', 'S', 'U', 'R', 'R', '0', '1'};
constexpr uint32_t kCkptWidth[4] = {256, 512, 512, 6};
}  // namespace

size_t rs_surrogate_checkpoint_bytes(void) { return sizeof(CkptHeader) + rs_surrogate_blob_bytes(); }

rs_status rs_surrogate_save(rs_ctx* c, const float* blob, void* host, size_t host_bytes) {
    if (!c) return RS_EINVAL;
    if (!blob || !host) return fail(c, RS_EINVAL, "blob and host are required");
    if (host_bytes < rs_surrogate_checkpoint_bytes())
        return fail(c, RS_EINVAL, "host buffer has %zu bytes, needs %zu", host_bytes, rs_surrogate_checkpoint_bytes());
    cudaSetDevice(c->device);
    unsigned char* out = static_cast<unsigned char*>(host);
    const size_t nb = rs_surrogate_blob_bytes();
    cudaError_t e = cudaMemcpyAsync(out + sizeof(CkptHeader), blob, nb, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "rs_surrogate_save");
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kCkptMagic, sizeof(h.magic));
    h.version = 1;
    memcpy(h.width, kCkptWidth, sizeof(h.width));
    h.dtype = 0;
    int32_t t = 0;                // counters: [0] minibatch position, [1] AdamW's t
    memcpy(&t, out + sizeof(CkptHeader) + (size_t)rs_surrogate_blob_offset(10) * sizeof(float) + sizeof(int32_t),
           sizeof(t));
    h.step = t;
    h.blob_bytes = nb;
    memcpy(out, &h, sizeof(h));
    return RS_OK;
}

rs_status rs_surrogate_restore(rs_ctx* c, float* blob, const void* host, size_t host_bytes) {
    if (!c) return RS_EINVAL;
    if (!blob || !host) return fail(c, RS_EINVAL, "blob and host are required");
    if ((uintptr_t)blob % 256) return fail(c, RS_EINVAL, "blob must be 256-byte aligned");
    if (host_bytes < sizeof(CkptHeader)) return fail(c, RS_EINVAL, "not a surrogate checkpoint (too short)");
    CkptHeader h;
    memcpy(&h, host, sizeof(h));
    if (memcmp(h.magic, kCkptMagic, sizeof(h.magic)) != 0) return fail(c, RS_EINVAL, "not a surrogate checkpoint");
    if (h.version != 1) return fail(c, RS_EINVAL, "checkpoint format version %u, expected 1", h.version);
    if (memcmp(h.width, kCkptWidth, sizeof(h.width)) != 0 || h.dtype != 0)
        return fail(c, RS_EINVAL, "checkpoint of another network shape or element type");
    const size_t nb = rs_surrogate_blob_bytes();
    if (h.blob_bytes != nb || host_bytes < sizeof(CkptHeader) + nb)
        return fail(c, RS_EINVAL, "checkpoint blob of %llu bytes, expected %zu", (unsigned long long)h.blob_bytes, nb);
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemcpyAsync(blob, static_cast<const unsigned char*>(host) + sizeof(CkptHeader), nb,
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_surrogate_restore");
}

}  // extern "C"

namespace {

// The fallback's scratch inside the caller's workspace, sized for the whole batch (every
// program selected), 256-byte aligned pieces; base == nullptr only measures.
rs_fallback_ws carve_fallback(void* base, const rs_batch* b, const rs_splits* sp) {
    rs_fallback_ws w{};
    char* c = (char*)base;
    size_t o = 0;
    auto take = [&](size_t n) -> void* {
        void* p = c ? (void*)(c + o) : nullptr;
        o += align256(n > 0 ? n : 1);
        return p;
    };
    const int64_t P = b->n_programs, S = sp->n_splits;
    const int64_t rows_cap = sp->n_test_rows > 0 ? sp->n_test_rows : S * (int64_t)b->max_versions;
    const size_t es = b->dtype == RS_F32 ? 4 : 8;
    w.totals = (long long*)take(8 * sizeof(long long));
    w.prog_map = (int32_t*)take((size_t)P * sizeof(int32_t));
    w.sub_prog = (int32_t*)take((size_t)P * sizeof(int32_t));
    w.sub_row_off = (int64_t*)take((size_t)(P + 1) * sizeof(int64_t));
    w.sub_x_off = (int64_t*)take((size_t)P * sizeof(int64_t));
    w.sub_feat_off = (int64_t*)take((size_t)(P + 1) * sizeof(int64_t));
    w.sub_split_off = (int64_t*)take((size_t)(P + 1) * sizeof(int64_t));
    w.sub_fw = (int32_t*)take((size_t)P * sizeof(int32_t));
    w.sX = take((size_t)b->x_elems * es);
    w.s_masks = (uint8_t*)take((size_t)b->n_rows);
    w.s_lt = (double*)take((size_t)b->n_rows * sizeof(double));
    w.s_cyc = (double*)take((size_t)b->n_rows * sizeof(double));
    w.s_train = (uint64_t*)take((size_t)S * sizeof(uint64_t));
    w.s_rec_off = (int64_t*)take((size_t)(S + 1) * sizeof(int64_t));
    w.s_code = (uint32_t*)take((size_t)rows_cap * sizeof(uint32_t));
    w.s_pred = (double*)take((size_t)rows_cap * RS_NOPT * sizeof(double));
    w.cv_ws_bytes = rs_cv_workspace_bytes(b, sp);
    w.cv_ws = take(w.cv_ws_bytes);
    w.bytes = o;
    return w;
}

}  // namespace

extern "C" {

size_t rs_pooled_workspace_bytes(const rs_batch* b) {
    if (rs_batch_problem(b, false) || b->max_feat > 512) return 0;
    return rs_pooled_workspace_bytes_impl(b->n_programs, b->max_feat);
}

rs_status rs_fit_pooled(rs_ctx* c, const rs_batch* b, const uint8_t* use_program, double lambda, int flags,
                        void* ws, size_t ws_bytes, double* coef, uint8_t* fit_status) {
    if (!c) return RS_EINVAL;
    rs_status s = check_batch(c, b, false);
    if (s != RS_OK) return s;
    if (b->max_feat > 512) return fail(c, RS_EINVAL, "pooled fits: max_feat <= 512");
    if (b->n_programs > 65535) return fail(c, RS_EINVAL, "pooled fits: at most 65,535 programs");
    if (!(lambda > 0.0) || !isfinite(lambda)) return fail(c, RS_EINVAL, "lambda must be finite and > 0");
    if (flags & ~RS_REFINE_X) return fail(c, RS_EINVAL, "flags: RS_REFINE_X only");
    if (!coef || !fit_status) return fail(c, RS_EINVAL, "coef and fit_status are required");
    if (!ws || (uintptr_t)ws % 256 != 0) return fail(c, RS_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    const size_t need = rs_pooled_workspace_bytes_impl(b->n_programs, b->max_feat);
    if (ws_bytes < need) return fail(c, RS_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, need);
    cudaSetDevice(c->device);
    cudaError_t e = rs_launch_fit_pooled(b, use_program, lambda, (flags & RS_REFINE_X) ? 1 : 0, ws, ws_bytes, coef,
                                         fit_status, c->dstatus, c->stream);
    if (e == cudaErrorNotSupported) return fail(c, RS_EUNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_fit_pooled");
}

rs_status rs_predict_pooled(rs_ctx* c, const rs_batch* b, const double* coef, const uint8_t* fit_status, int k,
                            double tau, int flags, uint32_t* rec_code, double* rec_pred, double* pred_all,
                            uint64_t* counters) {
    if (!c) return RS_EINVAL;
    rs_status s = check_batch(c, b, false);
    if (s != RS_OK) return s;
    if (b->max_feat > 512) return fail(c, RS_EINVAL, "pooled fits: max_feat <= 512");
    if (!coef || !fit_status || !rec_code) return fail(c, RS_EINVAL, "coef, fit_status and rec_code are required");
    if (k < 1 || k > RS_NOPT) return fail(c, RS_EINVAL, "k must be in 1..6");
    if (!(tau > 0.0) || !isfinite(tau)) return fail(c, RS_EINVAL, "tau must be finite and > 0");
    if (flags & ~RS_RANK_ALL) return fail(c, RS_EINVAL, "flags: RS_RANK_ALL only");
    cudaSetDevice(c->device);
    cudaError_t e = rs_launch_predict_pooled(b, coef, fit_status, k, log(tau), flags, rec_code, rec_pred, pred_all,
                                             (unsigned long long*)counters, c->dstatus, c->stream);
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_predict_pooled");
}

size_t rs_fallback_workspace_bytes(const rs_batch* b, const rs_splits* sp) {
    if (rs_batch_problem(b, true) || rs_splits_problem(sp)) return 0;
    return carve_fallback(nullptr, b, sp).bytes;
}

rs_status rs_surrogate_fallback(rs_ctx* c, const rs_batch* b, const rs_splits* sp, const uint8_t* used_fallback,
                                double lambda, int k, double tau, int flags, void* ws, size_t ws_bytes,
                                uint32_t* rec_code, double* rec_pred, int64_t* refit) {
    if (!c) return RS_EINVAL;
    rs_status s = check_batch(c, b, true);
    if (s == RS_OK) s = check_splits(c, sp);
    if (s != RS_OK) return s;
    if (!used_fallback || !rec_code) return fail(c, RS_EINVAL, "used_fallback and rec_code are required");
    if (k < 1 || k > RS_NOPT) return fail(c, RS_EINVAL, "k must be in 1..6");
    if (!(tau > 0.0) || !isfinite(tau)) return fail(c, RS_EINVAL, "tau must be finite and > 0");
    if (!(lambda >= 0.0) || !isfinite(lambda)) return fail(c, RS_EINVAL, "lambda must be finite and >= 0");
    if (flags & ~RS_RANK_ALL) return fail(c, RS_EINVAL, "flags: RS_RANK_ALL only");
    if (!ws || (uintptr_t)ws % 256 != 0) return fail(c, RS_EINVAL, "workspace must be non-NULL and 256-byte aligned");
    const size_t need = carve_fallback(nullptr, b, sp).bytes;
    if (ws_bytes < need) return fail(c, RS_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, need);
    const rs_fallback_ws w = carve_fallback(ws, b, sp);
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemsetAsync(w.totals, 0, 8 * sizeof(long long), c->stream);
    if (e == cudaSuccess) e = rs_launch_fallback_select(b, sp, used_fallback, w, c->stream);
    long long tot[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(tot, w.totals, sizeof(tot), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);     // the sub-batch's sizes
    if (e != cudaSuccess) return cuda_fail(c, e, "rs_surrogate_fallback (selection)");
    const int Q = (int)tot[0];
    if (Q > 0) {
        e = rs_launch_fallback_gather(b, sp, Q, w, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "rs_surrogate_fallback (gather)");
        rs_batch sb = *b;
        sb.n_programs = Q;
        sb.n_rows = tot[1];
        sb.x_elems = tot[2];
        sb.feat_total = tot[5];
        sb.row_offsets = w.sub_row_off;
        sb.feat_width = w.sub_fw;
        sb.x_offsets = w.sub_x_off;
        sb.feat_offsets = w.sub_feat_off;
        sb.X = w.sX;
        sb.masks = w.s_masks;
        sb.log_time = w.s_lt;
        sb.cycles = b->cycles ? w.s_cyc : nullptr;
        rs_splits ss = *sp;
        ss.n_splits = tot[3];
        ss.n_test_rows = tot[4];
        ss.split_offsets = w.sub_split_off;
        ss.train_masks = w.s_train;
        s = rs_cv_step(c, &sb, &ss, lambda, k, tau, flags, RS_GRAM_F64, w.cv_ws, w.cv_ws_bytes, w.s_rec_off,
                       w.s_code, w.s_pred, nullptr, nullptr);
        if (s != RS_OK) return s;
        e = rs_launch_fallback_merge(b, used_fallback, w, k, rec_code, rec_pred, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "rs_surrogate_fallback (merge)");
    }
    if (refit) {
        refit[0] = Q;
        refit[1] = tot[1];
    }
    return RS_OK;
}

size_t rs_cv_workspace_bytes(const rs_batch* b, const rs_splits* sp) {
    if (!b || !sp || b->n_programs < 1 || b->x_elems < 0) return 0;
    size_t z = align256((size_t)b->x_elems * sizeof(double));
    size_t k = align256((size_t)b->n_programs * RS_GRAM_LD * RS_GRAM_LD * sizeof(double));
    size_t f = align256(rs_fit_workspace_bytes(b, sp));
    size_t g = align256(rs_gram_workspace_bytes(b, RS_GRAM_BF16X3));
    return z + k + (f > g ? f : g);     // the Gram's scratch is free again when the fits start
}

rs_status rs_cv_step(rs_ctx* c, const rs_batch* b, const rs_splits* sp, double lambda, int k,
                     double tau, int flags, int precision, void* ws, size_t ws_bytes,
                     int64_t* rec_offsets, uint32_t* rec_code, double* rec_pred,
                     double* pred_all, uint64_t* counters) {
    if (!c) return RS_EINVAL;
    rs_status s = check_batch(c, b, true);
    if (s != RS_OK) return s;
    if (!ws) return fail(c, RS_EINVAL, "workspace is NULL");
    if ((uintptr_t)ws % 256 != 0) return fail(c, RS_EINVAL, "workspace must be 256-byte aligned");
    s = check_splits(c, sp);
    if (s != RS_OK) return s;
    const size_t need = rs_cv_workspace_bytes(b, sp);
    if (ws_bytes < need) return fail(c, RS_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, need);
    double* Z = (double*)ws;
    const size_t zbytes = align256((size_t)b->x_elems * sizeof(double));
    const size_t kbytes = align256((size_t)b->n_programs * RS_GRAM_LD * RS_GRAM_LD * sizeof(double));
    double* K = (double*)((char*)ws + zbytes);
    void* fws = (char*)ws + zbytes + kbytes;
    const size_t fbytes = ws_bytes - zbytes - kbytes;
    rs_batch zb = *b;
    zb.X = Z;
    zb.dtype = RS_F64;
    if (flags & RS_MODEL_IBK) {
        if (precision != RS_GRAM_F64 && precision != RS_GRAM_DIST2)
            return fail(c, RS_EINVAL, "RS_MODEL_IBK takes precision RS_GRAM_F64 or RS_GRAM_DIST2");
        precision = RS_GRAM_DIST2;
    }
    if (precision != RS_GRAM_F64 && precision != RS_GRAM_DIST2 && precision != RS_GRAM_BF16X3)
        return fail(c, RS_EINVAL, "unknown precision %d", precision);
    if (!rec_offsets) return fail(c, RS_EINVAL, "rec_offsets is NULL");
    rs_fit_args a;
    s = predict_args(c, &zb, K, sp, lambda, nullptr, k, tau, flags, RS_FORM_BATCHED, fws, fbytes,
                     rec_offsets, rec_code, rec_pred, pred_all, counters, a);
    if (s != RS_OK) return s;
    cudaSetDevice(c->device);
    cudaError_t e = cudaSuccess;
    if (!c->side || !c->fork || !c->join || precision == RS_GRAM_BF16X3) {
        // one stream, in order: the tensor-core Gram's scratch is the fit workspace, which the
        // planning fills afterwards
        s = rs_standardize(c, b, Z, nullptr, nullptr);
        if (s == RS_OK) s = rs_gram(c, &zb, precision, K, fws, fbytes);
        if (s != RS_OK) return s;
        e = rs_launch_rec_offsets(&zb, sp, rec_offsets, c->scan, c->dstatus, c->stream);
        if (e == cudaSuccess) e = rs_launch_fit_predict(a, c->stream);
        return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_cv_step");
    }
    // The planning (row offsets, pair tables, fit plan, bucketing) reads only masks, times and
    // splits: on the side stream it runs beside the standardization and the Gram (which use
    // no part of the fit workspace), and the solvers wait for both.
    e = cudaEventRecord(c->fork, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->fork, 0);
    if (e == cudaSuccess) e = rs_launch_rec_offsets(&zb, sp, rec_offsets, c->scan, c->dstatus, c->side);
    if (e == cudaSuccess) {
        a.phase = 1;
        e = rs_launch_fit_predict(a, c->side);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->join, c->side);
    if (e != cudaSuccess) return cuda_fail(c, e, "rs_cv_step (planning)");
    s = rs_standardize(c, b, Z, nullptr, nullptr);
    if (s == RS_OK) s = rs_gram(c, &zb, precision, K, fws, fbytes);
    e = cudaStreamWaitEvent(c->stream, c->join, 0);   // joined whatever happened above
    if (s != RS_OK) return s;
    if (e != cudaSuccess) return cuda_fail(c, e, "rs_cv_step (join)");
    a.phase = 2;
    e = rs_launch_fit_predict(a, c->stream);
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_cv_step");
}


// ---- Table 2 transfer ----------------------------------------------------------------------------
namespace {
struct TransferWs {
    double *ZA, *ZB, *mu, *sigma, *KA, *Kx, *fit;
    void* m5;
    int64_t* iota;
    size_t bytes;
};

int transfer_runs(const rs_groups* g) { return g ? g->max_runs : 1; }

TransferWs transfer_carve(void* base, const rs_batch* train, const rs_batch* test, const rs_groups* g, int flags) {
    TransferWs w{};
    char* c = (char*)base;
    size_t o = 0;
    auto take = [&](size_t b) { char* p = c ? c + o : nullptr; o += align256(b); return p; };
    const size_t Q = (size_t)test->n_programs;
    const size_t ld = (size_t)RS_MAXV * transfer_runs(g);
    w.ZA = (double*)take((size_t)train->x_elems * sizeof(double));
    w.ZB = (double*)take((size_t)test->x_elems * sizeof(double));
    w.mu = (double*)take(Q * (size_t)train->max_feat * sizeof(double));
    w.sigma = (double*)take(Q * (size_t)train->max_feat * sizeof(double));
    w.KA = (double*)take(Q * ld * ld * sizeof(double));
    w.Kx = (double*)take(Q * RS_MAXV * ld * sizeof(double));
    w.fit = (double*)take(rs_transfer_fit_bytes((int64_t)Q));
    w.m5 = (flags & RS_MODEL_M5P) ? take(Q * RS_NOPT * rs_m5p_tree_bytes()) : nullptr;
    w.iota = g ? nullptr : (int64_t*)take((Q + 1) * sizeof(int64_t));
    w.bytes = o;
    return w;
}
}  // namespace

size_t rs_transfer_workspace_bytes(const rs_batch* train, const rs_batch* test, const rs_groups* groups,
                                   int flags) {
    if (!train || !test || test->n_programs < 1 || train->x_elems < 0 || test->x_elems < 0 ||
        train->max_feat < 1 || (groups && (groups->max_runs < 1 || groups->max_runs > RS_MAXRUNS)))
        return 0;
    return transfer_carve(nullptr, train, test, groups, flags).bytes;
}

rs_status rs_transfer(rs_ctx* c, const rs_batch* train, const rs_batch* test, const rs_groups* groups,
                      double lambda, int k, double tau, int flags, int opt_mask, void* ws, size_t ws_bytes,
                      uint8_t* fit_status, uint32_t* rec_code, double* rec_pred, double* pred_all,
                      uint64_t* counters) {
    if (!c) return RS_EINVAL;
    rs_status s = check_batch(c, train, true);
    if (s == RS_OK) s = check_batch(c, test, true);
    if (s != RS_OK) return s;
    if (groups) {
        if (groups->n_groups != test->n_programs)
            return fail(c, RS_EINVAL, "groups->n_groups must equal the test set's n_programs");
        if (groups->max_runs < 1 || groups->max_runs > RS_MAXRUNS)
            return fail(c, RS_EINVAL, "groups->max_runs must be in 1..%d", RS_MAXRUNS);
        if (!groups->group_offsets) return fail(c, RS_EINVAL, "groups->group_offsets is NULL");
    } else if (train->n_programs != test->n_programs) {
        return fail(c, RS_EINVAL, "without groups the training and test sets hold the same number of programs");
    }
    if (!(lambda >= 0.0) || !isfinite(lambda)) return fail(c, RS_EINVAL, "lambda must be finite and >= 0");
    if (k < 1 || k > RS_NOPT) return fail(c, RS_EINVAL, "k must be in 1..6");
    if (!(tau > 0.0) || !isfinite(tau)) return fail(c, RS_EINVAL, "tau must be finite and > 0");
    if (flags & ~(RS_RANK_ALL | RS_MODEL_IBK | RS_MODEL_M5P))
        return fail(c, RS_EINVAL, "flags: RS_RANK_ALL, RS_MODEL_IBK and RS_MODEL_M5P only");
    if ((flags & RS_MODEL_IBK) && (flags & RS_MODEL_M5P)) return fail(c, RS_EINVAL, "one model: IBK or M5P");
    if ((flags & RS_MODEL_M5P) && train->max_feat > rs_m5p_max_feat())
        return fail(c, RS_EUNSUPPORTED, "RS_MODEL_M5P takes at most %d features", rs_m5p_max_feat());
    if (opt_mask < 0 || opt_mask > 63) return fail(c, RS_EINVAL, "opt_mask must be in 0..63");
    if (!rec_code) return fail(c, RS_EINVAL, "rec_code is required");
    if (!ws) return fail(c, RS_EINVAL, "workspace is NULL");
    if ((uintptr_t)ws % 256 != 0) return fail(c, RS_EINVAL, "workspace must be 256-byte aligned");
    const size_t need = rs_transfer_workspace_bytes(train, test, groups, flags);
    if (ws_bytes < need) return fail(c, RS_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, need);
    TransferWs w = transfer_carve(ws, train, test, groups, flags);
    cudaSetDevice(c->device);
    const bool ibk = (flags & RS_MODEL_IBK) != 0;
    const bool m5p = (flags & RS_MODEL_M5P) != 0;
    const int Q = test->n_programs;
    const int max_runs = transfer_runs(groups);
    const int ld = RS_MAXV * max_runs;
    const int stride = train->max_feat;
    cudaError_t e = cudaSuccess;
    const int64_t* goff = groups ? groups->group_offsets : w.iota;
    if (!groups) e = rs_launch_iota64(w.iota, (int64_t)Q + 1, c->stream);
    if (e == cudaSuccess)
        e = rs_launch_transfer_standardize(train, test, goff, max_runs, stride, w.ZA, w.ZB, w.mu, w.sigma,
                                           c->dstatus, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "rs_transfer (standardize)");
    rs_batch za = *train, zb = *test;
    za.X = w.ZA;
    za.dtype = RS_F64;
    zb.X = w.ZB;
    zb.dtype = RS_F64;
    if (!m5p) {                 // the model tree reads the standardized rows themselves
        e = rs_launch_transfer_blocks(&za, &zb, goff, max_runs, stride, ld, ibk ? nullptr : w.KA, w.Kx, ibk ? 1 : 0,
                                      c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "rs_transfer (blocks)");
    }
    rs_transfer_args t{};
    t.Q = Q;
    t.group_off = goff;
    t.max_runs = max_runs;
    t.n_runs = train->n_programs;
    t.stat_stride = stride;
    t.a_row_offsets = train->row_offsets;
    t.a_feat_width = train->feat_width;
    t.a_masks = train->masks;
    t.a_log_time = train->log_time;
    t.b_row_offsets = test->row_offsets;
    t.b_feat_width = test->feat_width;
    t.b_masks = test->masks;
    t.b_log_time = test->log_time;
    t.KA = w.KA;
    t.Kx = w.Kx;
    t.ld = ld;
    t.lambda = lambda;
    t.ibk = ibk ? 1 : 0;
    t.opt_mask = opt_mask;
    t.k = k;
    t.log_tau = log(tau);   // host libm, as in rs_predict_rank
    t.flags = flags;
    t.fit_status = fit_status;
    t.fit_ws = w.fit;
    t.m5p = m5p ? 1 : 0;
    t.m5_ws = w.m5;
    t.ZA = w.ZA;
    t.a_x_offsets = train->x_offsets;
    t.ZB = w.ZB;
    t.b_x_offsets = test->x_offsets;
    t.rec_code = rec_code;
    t.rec_pred = rec_pred;
    t.pred_all = pred_all;
    t.counters = (unsigned long long*)counters;
    t.dstatus = c->dstatus;
    e = rs_launch_transfer(t, c->stream);
    return e == cudaSuccess ? RS_OK : cuda_fail(c, e, "rs_transfer");
}

// ---- CUDA graph of the whole step -------------------------------------------------------------
struct rs_graph {
    rs_ctx* ctx;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

rs_status rs_cv_graph_create(rs_ctx* c, const rs_batch* b, const rs_splits* sp, double lambda, int k,
                             double tau, int flags, int precision, void* ws, size_t ws_bytes,
                             int64_t* rec_offsets, uint32_t* rec_code, double* rec_pred, double* pred_all,
                             uint64_t* counters, rs_graph** out) {
    if (!c || !out) return RS_EINVAL;
    *out = nullptr;
    if (c->profiling) return fail(c, RS_EINVAL, "turn profiling off before capturing a graph");
    cudaSetDevice(c->device);
    cudaStream_t orig = c->stream, cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(c, e, "rs_cv_graph_create");
    c->stream = cap;
    // one eager pass first: function attributes and driver entry points are set up outside
    // the capture, and argument errors are reported before anything is recorded
    rs_status s = rs_cv_step(c, b, sp, lambda, k, tau, flags, precision, ws, ws_bytes, rec_offsets, rec_code,
                             rec_pred, pred_all, counters);
    if (s == RS_OK) {
        e = cudaStreamSynchronize(cap);
        if (e != cudaSuccess) s = cuda_fail(c, e, "rs_cv_graph_create (eager pass)");
    }
    cudaGraph_t g = nullptr;
    if (s == RS_OK) {
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) s = cuda_fail(c, e, "cudaStreamBeginCapture");
    }
    if (s == RS_OK) {
        rs_status s2 = rs_cv_step(c, b, sp, lambda, k, tau, flags, precision, ws, ws_bytes, rec_offsets,
                                  rec_code, rec_pred, pred_all, counters);
        e = cudaStreamEndCapture(cap, &g);
        if (s2 != RS_OK) s = s2;
        else if (e != cudaSuccess) s = cuda_fail(c, e, "cudaStreamEndCapture");
    }
    c->stream = orig;
    cudaStreamDestroy(cap);
    if (s != RS_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    rs_graph* r = new (std::nothrow) rs_graph{c, g, ex};
    if (!r) {
        cudaGraphExecDestroy(ex);
        cudaGraphDestroy(g);
        return RS_ENOMEM;
    }
    *out = r;
    return RS_OK;
}

rs_status rs_cv_graph_launch(rs_graph* g) {
    if (!g) return RS_EINVAL;
    cudaSetDevice(g->ctx->device);
    cudaError_t e = cudaGraphLaunch(g->exec, g->ctx->stream);
    return e == cudaSuccess ? RS_OK : cuda_fail(g->ctx, e, "rs_cv_graph_launch");
}

rs_status rs_cv_graph_destroy(rs_graph* g) {
    if (!g) return RS_EINVAL;
    cudaSetDevice(g->ctx->device);
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return RS_OK;
}

// ---- autotuner --------------------------------------------------------------------------------
}  // extern "C"

// Times the tensor-core Gram of this batch (raw counters: standardized into the workspace first,
// laid out as rs_cv_step does) for the four tile configurations and keeps the fastest for the
// batch's padded width.  times_ms (nullable) gets the four times in configuration order
// (64-column whole-K, 32 whole, 64 split, 32 split); *choice the configuration kept.
static rs_status rs_autotune_gram_impl(rs_ctx* c, const rs_batch* b, void* ws, size_t ws_bytes, float* times_ms,
                                       int* choice) {
    rs_status s = check_batch(c, b, true);
    if (s != RS_OK) return s;
    if (b->n_programs > 65535) return fail(c, RS_EINVAL, "the tensor-core Gram takes at most 65535 programs per call");
    const size_t zbytes = align256((size_t)b->x_elems * sizeof(double));
    const size_t kbytes = align256((size_t)b->n_programs * RS_GRAM_LD * RS_GRAM_LD * sizeof(double));
    const size_t gneed = rs_gram_tc_workspace_bytes(b->n_programs, b->max_feat);
    if (!ws || (uintptr_t)ws % 256 || ws_bytes < zbytes + kbytes + gneed)
        return fail(c, RS_ENOMEM, "autotuning the Gram needs %zu bytes of workspace", zbytes + kbytes + gneed);
    double* Z = (double*)ws;
    double* K = (double*)((char*)ws + zbytes);
    void* gws = (char*)ws + zbytes + kbytes;
    const size_t gbytes = ws_bytes - zbytes - kbytes;
    s = rs_standardize(c, b, Z, nullptr, nullptr);
    if (s != RS_OK) return s;
    rs_batch zb = *b;
    zb.X = Z;
    zb.dtype = RS_F64;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int keep = 0;
    cudaError_t e = cudaSuccess;
    for (int cfg = 0; cfg < 4 && e == cudaSuccess; ++cfg) {
        float ms = 0.f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            cudaEventRecord(e0, c->stream);
            e = rs_launch_gram_bf16x3_ws(&zb, K, gws, gbytes, c->dstatus, c->stream, (cfg & 1) ? 32 : 64,
                                         (cfg & 2) ? 3 : 1);
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);      // the last run is the one kept
        }
        if (times_ms) times_ms[cfg] = ms;
        if (ms < best) {
            best = ms;
            keep = cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(c, e, "rs_autotune_gram");
    c->gram_cfg[gram_slot(b->max_feat)] = (uint8_t)keep;
    if (choice) *choice = keep;
    return RS_OK;
}

extern "C" {

rs_status rs_autotune_gram(rs_ctx* c, const rs_batch* b, void* ws, size_t ws_bytes, float* times_ms, int* choice) {
    if (!c) return RS_EINVAL;
    cudaSetDevice(c->device);
    return rs_autotune_gram_impl(c, b, ws, ws_bytes, times_ms, choice);
}

rs_status rs_get_gram_tuning(const rs_ctx* c, int feat_width, int* tile_n, int* ksplit) {
    if (!c || feat_width < 1 || feat_width > 4096) return RS_EINVAL;
    const int cfg = c->gram_cfg[gram_slot(feat_width)];
    if (tile_n) *tile_n = (cfg & 1) ? 32 : 64;
    if (ksplit) *ksplit = (cfg & 2) ? 3 : 1;
    return RS_OK;
}

rs_status rs_set_gram_tuning(rs_ctx* c, int feat_width, int tile_n, int ksplit) {
    if (!c) return RS_EINVAL;
    if (feat_width < 1 || feat_width > 4096) return fail(c, RS_EINVAL, "feat_width must be in 1..4096");
    if ((tile_n != 32 && tile_n != 64) || (ksplit != 1 && ksplit != 3))
        return fail(c, RS_EINVAL, "tile_n must be 32 or 64 and ksplit 1 or 3");
    c->gram_cfg[gram_slot(feat_width)] = (uint8_t)((tile_n == 32 ? 1 : 0) | (ksplit == 3 ? 2 : 0));
    return RS_OK;
}

rs_status rs_autotune(rs_ctx* c, const rs_batch* b, const rs_splits* sp, double lambda, int k, double tau,
                      int flags, int precision, void* ws, size_t ws_bytes, int64_t* rec_offsets,
                      uint32_t* rec_code, double* rec_pred, float* times_ms, int* n_times) {
    if (!c) return RS_EINVAL;
    cudaSetDevice(c->device);
    const int splits_c[5] = {4, 5, 6, 7, 8};
    const int waves_c[3] = {8, 16, 32};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (precision == RS_GRAM_BF16X3) {          // the Gram's tiles first, on this batch
        rs_status gs = rs_autotune_gram_impl(c, b, ws, ws_bytes, nullptr, nullptr);
        if (gs != RS_OK) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return gs;
        }
    }
    float best = 1e30f;
    int bs = c->tune_split, bw = c->tune_rank_waves, bo = c->tune_order, idx = 0;
    rs_status s = RS_OK;
    for (int o = 0; o < 2 && s == RS_OK; ++o)
        for (int i = 0; i < 5 && s == RS_OK; ++i)
            for (int w = 0; w < 3 && s == RS_OK; ++w) {
                c->tune_split = splits_c[i];
                c->tune_rank_waves = waves_c[w];
                c->tune_order = o;
                float ms = 0.f;
                for (int rep = 0; rep < 2 && s == RS_OK; ++rep) {
                    cudaEventRecord(e0, c->stream);
                    s = rs_cv_step(c, b, sp, lambda, k, tau, flags, precision, ws, ws_bytes, rec_offsets, rec_code,
                                   rec_pred, nullptr, nullptr);
                    cudaEventRecord(e1, c->stream);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&ms, e0, e1);      // the second run is the one kept
                }
                if (times_ms && n_times && idx < *n_times) times_ms[idx] = ms;
                ++idx;
                if (s == RS_OK && ms < best) {
                    best = ms;
                    bs = splits_c[i];
                    bw = waves_c[w];
                    bo = o;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tune_split = bs;
    c->tune_rank_waves = bw;
    c->tune_order = bo;
    if (n_times) *n_times = idx;
    return s;
}

rs_status rs_get_tuning(const rs_ctx* c, int* solve_split, int* rank_waves, int* solve_order) {
    if (!c) return RS_EINVAL;
    if (solve_split) *solve_split = c->tune_split;
    if (rank_waves) *rank_waves = c->tune_rank_waves;
    if (solve_order) *solve_order = c->tune_order;
    return RS_OK;
}

rs_status rs_set_tuning(rs_ctx* c, int solve_split, int rank_waves, int solve_order) {
    if (!c) return RS_EINVAL;
    if (solve_split < 4 || solve_split > 8) return fail(c, RS_EINVAL, "solve_split must be in 4..8");
    if (rank_waves != 8 && rank_waves != 16 && rank_waves != 32)
        return fail(c, RS_EINVAL, "rank_waves must be 8, 16 or 32");
    if (solve_order != 0 && solve_order != 1) return fail(c, RS_EINVAL, "solve_order must be 0 or 1");
    c->tune_split = solve_split;
    c->tune_rank_waves = rank_waves;
    c->tune_order = solve_order;
    return RS_OK;
}

}  // extern "C"
