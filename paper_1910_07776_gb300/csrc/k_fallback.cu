// k_fallback.cu -- the plain predictor as the learned surrogate's fallback: the programs with
// a row that the surrogate flagged out of distribution are gathered into a sub-batch, run
// through the plain batched pass (rs_cv_step), and each flagged row takes the plain ranking
// of its version.  Three kernels: selection (which programs, and the sub-batch's offsets),
// gather (the sub-batch's inputs and splits), merge (the plain results into the surrogate's
// outputs).  The surrogate is not in the paper; the plain pass is its Sec. 2 / Sec. 3.4 method.
#include "rs_internal.cuh"

namespace {

constexpr int kSelThreads = 1024;
constexpr int kTotals = 6;   // programs, rows, x elements, splits, test rows, features

// Block-wide exclusive scan of kTotals int64 values per thread; returns the block totals.
__device__ void scan_totals(long long (&v)[kTotals], long long* wsum, long long* total) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    long long incl[kTotals];
#pragma unroll
    for (int q = 0; q < kTotals; ++q) {
        incl[q] = v[q];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, incl[q], d);
            if (lane >= d) incl[q] += y;
        }
        if (lane == 31) wsum[q * 32 + warp] = incl[q];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < kTotals; ++q) {
            long long w = wsum[q * 32 + lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += y;
            }
            wsum[q * 32 + lane] = w;
            if (lane == 31) total[q] = w;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kTotals; ++q) v[q] = incl[q] - v[q] + (warp > 0 ? wsum[q * 32 + warp - 1] : 0ll);
}

// One block.  Program p is selected when one of its rows has used_fallback set.  Per selected
// program q (in program order): prog_map[p] = q, sub_prog[q] = p, and the sub-batch's row,
// X-element, split and feature offsets; totals[0..5] = programs, rows, X elements, splits,
// test rows of those splits, features.
__global__ void __launch_bounds__(kSelThreads)
fallback_select_kernel(int P, const int64_t* __restrict__ row_off, const int32_t* __restrict__ fw,
                       const int64_t* __restrict__ split_off, const uint64_t* __restrict__ train,
                       const uint8_t* __restrict__ used, int32_t* prog_map, int32_t* sub_prog,
                       int64_t* sub_row_off, int64_t* sub_x_off, int64_t* sub_feat_off, int64_t* sub_split_off,
                       int32_t* sub_fw, long long* totals) {
    __shared__ long long wsum[kTotals * 32];
    __shared__ long long total[kTotals];
    const int tid = threadIdx.x;
    const int chunk = (P + kSelThreads - 1) / kSelThreads;
    const int p0 = tid * chunk, p1 = p0 + chunk < P ? p0 + chunk : P;
    auto measure = [&](int p, long long (&c)[kTotals]) -> bool {
        const int64_t r0 = row_off[p], r1 = row_off[p + 1];
        bool any = false;
        for (int64_t r = r0; r < r1 && !any; ++r) any = used[r] != 0;
        if (!any) return false;
        const int V = (int)(r1 - r0);
        const uint64_t full = rs_full_mask(V);
        long long trows = 0;
        for (int64_t s = split_off[p]; s < split_off[p + 1]; ++s) trows += V - __popcll(train[s] & full);
        c[0] = 1;
        c[1] = V;
        c[2] = (long long)V * fw[p];
        c[3] = split_off[p + 1] - split_off[p];
        c[4] = trows;
        c[5] = fw[p];
        return true;
    };
    long long acc[kTotals] = {0, 0, 0, 0, 0, 0};
    for (int p = p0; p < p1; ++p) {
        long long c[kTotals];
        if (measure(p, c))
#pragma unroll
            for (int q = 0; q < kTotals; ++q) acc[q] += c[q];
    }
    scan_totals(acc, wsum, total);
    for (int p = p0; p < p1; ++p) {
        long long c[kTotals];
        if (!measure(p, c)) {
            prog_map[p] = -1;
            continue;
        }
        const int q = (int)acc[0];
        prog_map[p] = q;
        sub_prog[q] = p;
        sub_row_off[q] = acc[1];
        sub_x_off[q] = acc[2];
        sub_split_off[q] = acc[3];
        sub_feat_off[q] = acc[5];
        sub_fw[q] = fw[p];
#pragma unroll
        for (int x = 0; x < kTotals; ++x) acc[x] += c[x];
    }
    if (tid == 0) {
        const int Q = (int)total[0];
        sub_row_off[Q] = total[1];
        sub_split_off[Q] = total[3];
        sub_feat_off[Q] = total[5];
#pragma unroll
        for (int q = 0; q < kTotals; ++q) totals[q] = total[q];
    }
}

// One block per selected program: its X rows (4- or 8-byte elements, copied as 4-byte words),
// masks, log times, cycles and its splits' train masks, into the sub-batch's layout.
__global__ void __launch_bounds__(256)
fallback_gather_kernel(int es, const int64_t* __restrict__ row_off, const int32_t* __restrict__ fw,
                       const int64_t* __restrict__ x_off, const void* __restrict__ X, const uint8_t* __restrict__ masks,
                       const double* __restrict__ lt, const double* __restrict__ cyc,
                       const int64_t* __restrict__ split_off, const uint64_t* __restrict__ train,
                       const int32_t* __restrict__ sub_prog, const int64_t* __restrict__ sub_row_off,
                       const int64_t* __restrict__ sub_x_off, const int64_t* __restrict__ sub_split_off,
                       void* sX, uint8_t* s_masks, double* s_lt, double* s_cyc, uint64_t* s_train) {
    const int q = blockIdx.x;
    const int p = sub_prog[q];
    const int64_t r0 = row_off[p], V = row_off[p + 1] - r0;
    const int64_t words = V * fw[p] * (es / 4);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(X) + x_off[p] * (es / 4);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sX) + sub_x_off[q] * (es / 4);
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    const int64_t d0 = sub_row_off[q];
    for (int64_t v = threadIdx.x; v < V; v += blockDim.x) {
        s_masks[d0 + v] = masks[r0 + v];
        s_lt[d0 + v] = lt[r0 + v];
        if (cyc) s_cyc[d0 + v] = cyc[r0 + v];
    }
    const int64_t s0 = split_off[p], ns = split_off[p + 1] - s0, t0 = sub_split_off[q];
    for (int64_t s = threadIdx.x; s < ns; s += blockDim.x) s_train[t0 + s] = train[s0 + s];
}

// Row i of the full batch with used[i] set: its version v of program p takes the plain pass's
// ranking from the first split of p (in the sub-batch) that tests v.
__global__ void __launch_bounds__(256)
fallback_merge_kernel(int P, int64_t n_rows, const int64_t* __restrict__ row_off, const uint8_t* __restrict__ used,
                      const int32_t* __restrict__ prog_map, const int64_t* __restrict__ sub_split_off,
                      const uint64_t* __restrict__ s_train, const int64_t* __restrict__ s_rec_off,
                      const uint32_t* __restrict__ s_code, const double* __restrict__ s_pred, int k,
                      uint32_t* rec_code, double* rec_pred, unsigned long long* merged) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool done = false;
    if (i < n_rows && used[i]) {
        const int p = rs_find_segment(row_off, P, i);
        const int q = prog_map[p];
        const int v = (int)(i - row_off[p]);
        const uint64_t full = rs_full_mask((int)(row_off[p + 1] - row_off[p]));
        if (q >= 0)
            for (int64_t s = sub_split_off[q]; s < sub_split_off[q + 1]; ++s) {
                const uint64_t T = s_train[s] & full;
                if ((T >> v) & 1) continue;
                const int64_t r = s_rec_off[s] + __popcll(~T & full & ((1ull << v) - 1ull));
                rec_code[i] = s_code[r];
                if (rec_pred)
                    for (int x = 0; x < k; ++x) rec_pred[i * k + x] = s_pred[r * k + x];
                done = true;
                break;
            }
    }
    const unsigned c = __reduce_add_sync(0xffffffffu, done ? 1u : 0u);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(merged, (unsigned long long)c);
}

}  // namespace

cudaError_t rs_launch_fallback_select(const rs_batch* b, const rs_splits* sp, const uint8_t* used,
                                      const rs_fallback_ws& w, cudaStream_t st) {
    fallback_select_kernel<<<1, kSelThreads, 0, st>>>(b->n_programs, b->row_offsets, b->feat_width,
                                                     sp->split_offsets, sp->train_masks, used, w.prog_map,
                                                     w.sub_prog, w.sub_row_off, w.sub_x_off, w.sub_feat_off,
                                                     w.sub_split_off, w.sub_fw, w.totals);
    return cudaGetLastError();
}

cudaError_t rs_launch_fallback_gather(const rs_batch* b, const rs_splits* sp, int Q, const rs_fallback_ws& w,
                                      cudaStream_t st) {
    if (Q < 1) return cudaSuccess;
    const int es = b->dtype == RS_F32 ? 4 : 8;
    fallback_gather_kernel<<<Q, 256, 0, st>>>(es, b->row_offsets, b->feat_width, b->x_offsets, b->X, b->masks,
                                              b->log_time, b->cycles, sp->split_offsets, sp->train_masks,
                                              w.sub_prog, w.sub_row_off, w.sub_x_off, w.sub_split_off, w.sX,
                                              w.s_masks, w.s_lt, b->cycles ? w.s_cyc : nullptr, w.s_train);
    return cudaGetLastError();
}

cudaError_t rs_launch_fallback_merge(const rs_batch* b, const uint8_t* used, const rs_fallback_ws& w, int k,
                                     uint32_t* rec_code, double* rec_pred, cudaStream_t st) {
    if (b->n_rows < 1) return cudaSuccess;
    const int64_t blocks = (b->n_rows + 255) / 256;
    fallback_merge_kernel<<<(unsigned)blocks, 256, 0, st>>>(b->n_programs, b->n_rows, b->row_offsets, used,
                                                            w.prog_map, w.sub_split_off, w.s_train, w.s_rec_off,
                                                            w.s_code, w.s_pred, k, rec_code, rec_pred,
                                                            reinterpret_cast<unsigned long long*>(w.totals + 6));
    return cudaGetLastError();
}
