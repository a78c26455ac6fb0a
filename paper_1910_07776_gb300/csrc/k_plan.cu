// A2 planning: the test rows of each split (version slots outside its train mask, Sec. 5)
// and their exclusive prefix sum, which indexes every per-row output.  Three launches:
// per-block counts + block sums, a single-block scan of the block sums, and the final
// per-block scan.  Integer work only; bit-exact by construction.
#include "rs_internal.cuh"

namespace {

constexpr int kScanThreads = 1024;
constexpr int kItems = 4;                       // splits per thread
constexpr int kPerBlock = kScanThreads * kItems;
constexpr int kMaxBlocks = kPerBlock;           // one block scans the block sums

// Block-wide exclusive scan of one int64 per thread; returns the block total in *total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
    __shared__ int64_t warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = (lane < kScanThreads / 32) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    const int64_t before = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
    *total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanThreads)
count_kernel(int P, const int64_t* row_off, const int64_t* split_off, const uint64_t* tm,
             int64_t S, int64_t* out, int64_t* block_sums) {
    const int64_t base = (int64_t)blockIdx.x * kPerBlock + (int64_t)threadIdx.x * kItems;
    int64_t local = 0;
    // one search for the thread's first split; its next splits are in the same program or
    // one of the programs after it
    int p = base < S ? rs_find_segment(split_off, P, base) : 0;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        const int64_t i = base + q;
        if (i < S) {
            while (p + 1 < P && split_off[p + 1] <= i) ++p;
            const int V = (int)(row_off[p + 1] - row_off[p]);
            const int64_t c = (V < 1 || V > RS_MAXV) ? 0 : V - __popcll(tm[i] & rs_full_mask(V));
            out[i] = c;
            local += c;
        }
    }
    int64_t total;
    (void)block_exclusive_scan(local, &total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
scan_block_sums_kernel(int64_t* block_sums, int nblocks, int64_t* grand_total) {
    int64_t v[kItems];
    int64_t local = 0;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        const int i = threadIdx.x * kItems + q;
        v[q] = i < nblocks ? block_sums[i] : 0;
        local += v[q];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(local, &total);
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        const int i = threadIdx.x * kItems + q;
        if (i < nblocks) block_sums[i] = run;
        run += v[q];
    }
    if (threadIdx.x == 0) *grand_total = total;
}

__global__ void __launch_bounds__(kScanThreads)
finish_kernel(int64_t* out, int64_t S, const int64_t* block_sums) {
    const int64_t base = (int64_t)blockIdx.x * kPerBlock + (int64_t)threadIdx.x * kItems;
    int64_t v[kItems];
    int64_t local = 0;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        const int64_t i = base + q;
        v[q] = i < S ? out[i] : 0;
        local += v[q];
    }
    int64_t total;
    int64_t run = block_exclusive_scan(local, &total) + block_sums[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        const int64_t i = base + q;
        if (i < S) out[i] = run;
        run += v[q];
    }
}

}  // namespace

size_t rs_rec_offsets_scratch_elems(int64_t n_splits) {
    return (size_t)((n_splits + kPerBlock - 1) / kPerBlock) + 1;
}

cudaError_t rs_launch_rec_offsets(const rs_batch* b, const rs_splits* s, int64_t* rec_offsets,
                                  int64_t* scratch, int* dstatus, cudaStream_t st) {
    (void)dstatus;
    const int64_t S = s->n_splits;
    const int64_t nb = (S + kPerBlock - 1) / kPerBlock;
    if (nb > kMaxBlocks) return cudaErrorInvalidValue;
    if (S == 0) return cudaMemsetAsync(rec_offsets, 0, sizeof(int64_t), st);
    count_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(b->n_programs, b->row_offsets,
                                                        s->split_offsets, s->train_masks, S,
                                                        rec_offsets, scratch);
    scan_block_sums_kernel<<<1, kScanThreads, 0, st>>>(scratch, (int)nb, rec_offsets + S);
    finish_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(rec_offsets, S, scratch);
    return cudaGetLastError();
}
