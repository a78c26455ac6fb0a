// rs_static.cu -- rs_cv_step_static: the whole cross-validation step with its scratch in a
// fixed device array owned by this library, for callers that cannot allocate device memory
// themselves (for example code running where every allocation must be made up front, or a
// host that hands the library only its own input and output buffers).  The paper has no
// counterpart; this is a deployment variant of rs_cv_step.
//
// g_rs_scratch below lives in device memory for as long as the library stays loaded (on
// every GPU that loads this module).  Host code must not use its name as an address: the
// device address is looked up with cudaGetSymbolAddress, with the device current, and cached
// per device together with the identity of the CUDA context it belongs to.  A context torn
// down and created again (cudaDeviceReset, for one) reloads the module, so a changed context
// identity triggers a fresh lookup instead of reusing a stale address.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cuda.h>

#include <mutex>

#include "rs_internal.cuh"

static __device__ __align__(256) unsigned char g_rs_scratch[RS_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
struct ScratchSlot {
    unsigned long long ctx_id;   // identity of the context the address was looked up in
    void* addr;
};
ScratchSlot g_slot[kMaxDevices] = {};
std::mutex g_scratch_mu;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// The unique identity of the current context, 0 if there is none or it cannot be read (then
// the address is looked up again on every call).  Called with g_scratch_mu held.
unsigned long long current_context_id() {
    static bool resolved = false;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!resolved) {
        resolved = true;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_current, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            get_id = nullptr;
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    unsigned long long id = 0;
    return get_id(ctx, &id) == CUDA_SUCCESS ? id : 0;
}

// The device address of g_rs_scratch on device `dev` (which must be current): looked up on
// the first call in each context of that device, cached afterwards.
cudaError_t scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long id = current_context_id();
    ScratchSlot& slot = g_slot[dev];
    if (!slot.addr || id == 0 || id != slot.ctx_id) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_rs_scratch);
        if (e != cudaSuccess) return e;
        slot.addr = p;
        slot.ctx_id = current_context_id();   // the lookup may have created the context
    }
    *out = slot.addr;
    return cudaSuccess;
}

rs_status say(char* buf, size_t len, rs_status code, const char* fmt, ...) {
    if (buf && len > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, len, fmt, ap);
        va_end(ap);
    }
    return code;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" rs_status rs_cv_step_static(void* cuda_stream, const rs_batch* b, const rs_splits* sp,
                                       double lambda, int k, double tau, int flags,
                                       int64_t* rec_offsets, uint32_t* rec_code, double* rec_pred,
                                       double* pred_all, uint64_t* counters, int* device_status,
                                       char* errbuf, size_t errbuf_len) {
    if (errbuf && errbuf_len) errbuf[0] = 0;
    // ---- arguments (the same rules as rs_cv_step)
    const char* why = rs_batch_problem(b, true);
    if (!why) why = rs_splits_problem(sp);
    if (why) return say(errbuf, errbuf_len, RS_EINVAL, "%s", why);
    if (!(lambda >= 0.0) || lambda > 1e300) return say(errbuf, errbuf_len, RS_EINVAL, "lambda must be >= 0");
    if (k < 1 || k > RS_NOPT) return say(errbuf, errbuf_len, RS_EINVAL, "k must be in 1..6");
    if (!(tau > 0.0) || tau > 1e300) return say(errbuf, errbuf_len, RS_EINVAL, "tau must be > 0");
    if (flags & ~RS_RANK_ALL) return say(errbuf, errbuf_len, RS_EINVAL, "only RS_RANK_ALL is accepted");
    if (!rec_offsets || !rec_code) return say(errbuf, errbuf_len, RS_EINVAL, "rec_offsets and rec_code are required");
    // sizes that cannot fit are refused before any product of them is formed
    if (b->x_elems > (int64_t)(RS_STATIC_SCRATCH_BYTES / sizeof(double)) ||
        b->n_programs > (int64_t)(RS_STATIC_SCRATCH_BYTES / (RS_GRAM_LD * RS_GRAM_LD * sizeof(double))) ||
        sp->n_splits > (int64_t)(RS_STATIC_SCRATCH_BYTES / (RS_NOPT * sizeof(uint32_t))))
        return say(errbuf, errbuf_len, RS_ENOMEM, "this batch cannot fit in the static scratch (%zu bytes)",
                   (size_t)RS_STATIC_SCRATCH_BYTES);

    // ---- scratch layout inside g_rs_scratch: status words | scan sums | Z | K | fit workspace
    const int64_t rows_cap = sp->n_test_rows > 0 ? sp->n_test_rows : sp->n_splits * (int64_t)b->max_versions;
    const size_t st_bytes = up256(RS_DST_INTS * sizeof(int));
    const size_t scan_bytes = up256(rs_rec_offsets_scratch_elems(sp->n_splits) * sizeof(int64_t));
    const size_t z_bytes = up256((size_t)b->x_elems * sizeof(double));
    const size_t k_bytes = up256((size_t)b->n_programs * RS_GRAM_LD * RS_GRAM_LD * sizeof(double));
    const size_t f_bytes = up256(rs_fit_workspace_bytes_impl(b->n_programs, sp->n_splits, sp->max_train, rows_cap));
    const size_t need = st_bytes + scan_bytes + z_bytes + k_bytes + f_bytes;
    if (need > (size_t)RS_STATIC_SCRATCH_BYTES)
        return say(errbuf, errbuf_len, RS_ENOMEM,
                   "this batch needs %zu bytes of scratch; the static scratch holds %zu bytes",
                   need, (size_t)RS_STATIC_SCRATCH_BYTES);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return say(errbuf, errbuf_len, RS_ECUDA, "no usable current device");
    char* base = nullptr;
    e = scratch_address(dev, (void**)&base);
    if (e != cudaSuccess)
        return say(errbuf, errbuf_len, RS_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int* dstatus = (int*)base;
    int64_t* scan = (int64_t*)(base + st_bytes);
    double* Z = (double*)(base + st_bytes + scan_bytes);
    double* K = (double*)(base + st_bytes + scan_bytes + z_bytes);
    void* fws = base + st_bytes + scan_bytes + z_bytes + k_bytes;

    // the status words carry over from the previous call: clear them
    e = cudaMemsetAsync(dstatus, 0, RS_DST_INTS * sizeof(int), st);
    if (e == cudaSuccess) e = rs_launch_standardize(b, Z, nullptr, nullptr, dstatus, st);
    rs_batch zb = *b;
    zb.X = Z;
    zb.dtype = RS_F64;
    if (e == cudaSuccess) e = rs_launch_gram_f64(&zb, K, dstatus, st);
    if (e == cudaSuccess) e = rs_launch_rec_offsets(&zb, sp, rec_offsets, scan, dstatus, st);
    if (e == cudaSuccess && sp->n_splits > 0) {
        rs_fit_args a;
        memset(&a, 0, sizeof(a));
        a.P = b->n_programs;
        a.row_offsets = b->row_offsets;
        a.feat_width = b->feat_width;
        a.x_offsets = b->x_offsets;
        a.Z = Z;
        a.masks = b->masks;
        a.log_time = b->log_time;
        a.K = K;
        a.S = sp->n_splits;
        a.split_offsets = sp->split_offsets;
        a.train_masks = sp->train_masks;
        a.lambda = lambda;
        a.k = k;
        a.log_tau = log(tau);
        a.flags = flags;
        a.form = RS_FORM_BATCHED;
        a.rec_offsets = rec_offsets;
        a.rec_code = rec_code;
        a.rec_pred = rec_pred;
        a.pred_all = pred_all;
        a.counters = (unsigned long long*)counters;
        a.dstatus = dstatus;
        a.queue = (unsigned int*)(dstatus + RS_DST_QUEUE);
        a.max_train = sp->max_train;
        a.rows_cap = rows_cap;
        a.workspace = fws;
        a.workspace_bytes = f_bytes;
        e = rs_launch_fit_predict(a, st);
    }
    if (e == cudaSuccess && device_status)
        e = cudaMemcpyAsync(device_status, dstatus, sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return say(errbuf, errbuf_len, RS_ECUDA, "launch: %s", cudaGetErrorString(e));
    return RS_OK;
}
