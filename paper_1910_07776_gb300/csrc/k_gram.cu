// K2 (FP64 form): per-program Gram block K_p = Z_p Z_p^T of the standardized feature
// vectors.  It is the only contraction of the method: every ridge fit of every split of
// program p reads its kernel entries K_p[v_a][v_b] from this block (dual form of the
// regression family of Sec. 3.4), so it is formed once per program, not once per fit.
//
// Grid: (program, chunk of 128 upper-triangle entries).  Entry e of a program (row-major
// over a <= b) is computed by thread e % 128 of chunk e / 128: one dot product over all F
// features, sequentially in f.  The program's rows come through shared memory in slices of
// 32 features, double-buffered with cp.async (the next slice lands while the current one is
// multiplied).  Every FMA is one of the V (V + 1) / 2 * F the block needs (no padding
// tiles); the mirrored entry is written by the same thread.
#include "rs_internal.cuh"

namespace {

constexpr int kGramThreads = 128;
constexpr int kGramSlice = 32;
constexpr int kGramLd = kGramSlice + 1;
constexpr int kGramChunks = (RS_MAXV * (RS_MAXV + 1) / 2 + kGramThreads - 1) / kGramThreads;

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Issues the copies of features [f0, f0 + w) of the program's V rows into buffer Zs.
__device__ __forceinline__ void stage_slice(double (*Zs)[kGramLd], const double* Zp, int V, int F, int f0, int w) {
    for (int t = threadIdx.x; t < V * kGramSlice; t += kGramThreads) {
        const int r = t / kGramSlice, c = t % kGramSlice;
        if (c < w) cp_async8(&Zs[r][c], Zp + (int64_t)r * F + f0 + c);
    }
}

// DIST = false: K_p[a][b] = sum_f z_a,f z_b,f (FMA chain).  DIST = true: the squared
// Euclidean distance sum_f (z_a,f - z_b,f)^2 with one rounding per subtraction, product and
// addition (no contraction), in ascending f -- the plain definition's arithmetic.
template <bool DIST>
__global__ void __launch_bounds__(kGramThreads)
gram_f64_kernel(int P, const int64_t* __restrict__ row_off, const int32_t* __restrict__ fw,
                const int64_t* __restrict__ xo, const double* __restrict__ Z,
                double* __restrict__ K, int* dstatus) {
    __shared__ double Zs[2][RS_MAXV][kGramLd];
    const int p = blockIdx.x;
    const int V = (int)(row_off[p + 1] - row_off[p]);
    if (V < 1 || V > RS_MAXV) {
        if (threadIdx.x == 0 && blockIdx.y == 0) rs_dev_flag(dstatus, RS_EDATA, p);
        return;
    }
    const int E = V * (V + 1) / 2;
    const int e = blockIdx.y * kGramThreads + threadIdx.x;
    if (blockIdx.y * kGramThreads >= E) return;
    const bool act = e < E;
    int a = 0, rem = e;                     // row a holds the V - a entries (a, a..V-1)
    while (act && rem >= V - a) {
        rem -= V - a;
        ++a;
    }
    const int b = a + rem;
    const int F = fw[p];
    const double* Zp = Z + xo[p];
    const int nsl = (F + kGramSlice - 1) / kGramSlice;
    stage_slice(Zs[0], Zp, V, F, 0, F < kGramSlice ? F : kGramSlice);
    cp_async_commit();
    double acc = 0.0;
    for (int k = 0; k < nsl; ++k) {
        const int f0 = k * kGramSlice;
        const int w = F - f0 < kGramSlice ? F - f0 : kGramSlice;
        if (k + 1 < nsl) {
            const int f1 = f0 + kGramSlice;
            stage_slice(Zs[(k + 1) & 1], Zp, V, F, f1, F - f1 < kGramSlice ? F - f1 : kGramSlice);
        }
        cp_async_commit();                  // (an empty group on the last slice)
        cp_async_wait1();                   // slice k has landed (for this thread's copies)
        __syncthreads();                    // ... and for everyone's
        if (act) {
            const double (*S)[kGramLd] = Zs[k & 1];
            if constexpr (DIST) {
#pragma unroll 8
                for (int c = 0; c < w; ++c) {
                    const double e = __dsub_rn(S[a][c], S[b][c]);
                    acc = __dadd_rn(acc, __dmul_rn(e, e));
                }
            } else {
#pragma unroll 8
                for (int c = 0; c < w; ++c) acc = fma(S[a][c], S[b][c], acc);
            }
        }
        __syncthreads();                    // buffer k & 1 is refilled in iteration k + 1
    }
    if (act) {
        double* Kp = K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
        Kp[a * RS_GRAM_LD + b] = acc;
        Kp[b * RS_GRAM_LD + a] = acc;
    }
}

// Blocks of a transfer problem q (Table 2), one thread per entry (kept for the IBK distance
// block, where the tiled form below measured slower).  Its training runs form one list of N versions
// (rs_group_layout); the rows are the list itself (CROSS false: the lower triangle u <= i of
// the group's Gram KA[q][i][u], ld x ld -- all that the fits read) or the versions of the
// test program q (CROSS true: Kx[q][t][u], 64 x ld).  Entry =
// sum_f z_i[f] z_u[f] (FMA chain), or with DIST sum_f (z_t[f] - z_u[f])^2 with unfused
// operations (the plain definition's arithmetic), ascending f.  One thread per entry; the
// rows come from L1 / L2.  Problems that fail the layout checks (reported by the
// standardization) are skipped.
template <bool CROSS, bool DIST>
__global__ void __launch_bounds__(128)
transfer_block_kernel(const int64_t* __restrict__ group_off, int max_runs, int64_t n_runs, int stat_stride,
                      const int64_t* __restrict__ a_row, const int32_t* __restrict__ a_fw,
                      const int64_t* __restrict__ a_xo, const double* __restrict__ ZA,
                      const int64_t* __restrict__ b_row, const int32_t* __restrict__ b_fw,
                      const int64_t* __restrict__ b_xo, const double* __restrict__ ZB, int ld,
                      double* __restrict__ out) {
    __shared__ int64_t rowx[RS_MAXV * RS_MAXRUNS];
    const int q = blockIdx.x;
    int start[RS_MAXRUNS + 1], F = 0;
    const int N = rs_group_layout(q, group_off, max_runs, n_runs, a_row, a_fw, b_fw, stat_stride, start, F);
    if (N < 0 || N > ld) return;
    const int VB = (int)(b_row[q + 1] - b_row[q]);
    if (CROSS && (VB < 1 || VB > RS_MAXV)) return;
    const int rows = CROSS ? VB : N;
    const int entries = CROSS ? rows * N : N * (N + 1) / 2;
    if ((int64_t)blockIdx.y * blockDim.x >= entries) return;
    const int64_t g0 = group_off[q];
    for (int u = threadIdx.x; u < N; u += blockDim.x) {
        int r = 0;
        while (u >= start[r + 1]) ++r;
        rowx[u] = a_xo[g0 + r] + (int64_t)(u - start[r]) * F;
    }
    __syncthreads();
    const int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= entries) return;
    int i, u;
    if constexpr (CROSS) {
        i = e / N;
        u = e - i * N;
    } else {                                   // e = i (i + 1) / 2 + u, u <= i
        i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (i * (i + 1) / 2 > e) --i;
        while ((i + 1) * (i + 2) / 2 <= e) ++i;
        u = e - i * (i + 1) / 2;
    }
    const double* zi = CROSS ? ZB + b_xo[q] + (int64_t)i * F : ZA + rowx[i];
    const double* zu = ZA + rowx[u];
    double acc = 0.0;
    for (int f = 0; f < F; ++f) {
        if constexpr (DIST) {
            const double d = __dsub_rn(__ldg(zi + f), __ldg(zu + f));
            acc = __dadd_rn(acc, __dmul_rn(d, d));
        } else {
            acc = fma(__ldg(zi + f), __ldg(zu + f), acc);
        }
    }
    const int64_t rows_ld = CROSS ? RS_MAXV : ld;
    out[((int64_t)q * rows_ld + i) * ld + u] = acc;
}

// Blocks of a transfer problem q (Table 2).  Its training runs form one list of N versions
// (rs_group_layout); the rows are the list itself (CROSS false: the lower triangle u <= i of
// the group's Gram KA[q][i][u], ld x ld -- all that the fits read) or the versions of the
// test program q (CROSS true: Kx[q][t][u], 64 x ld).  Entry = sum_f z_i[f] z_u[f] (FMA
// chain), or with DIST sum_f (z_t[f] - z_u[f])^2 with unfused operations (the plain
// definition's arithmetic), ascending f.  Problems that fail the layout checks (reported by
// the standardization) are skipped.  A block computes a 32 x 32 tile of entries (rows i0..,
// columns u0..; for the group's Gram only tiles with u0 <= i0, and entries u <= i), 16 x 16
// threads of 2 x 2 entries each.  The tile's rows come through shared memory in slices of 32
// features, one row per warp-row of lanes (coalesced); each entry sums its features in
// ascending order, one slice after another.
constexpr int kTT = 32;                      // tile edge
constexpr int kTS = 32;                      // features per slice
template <bool CROSS, bool DIST>
__global__ void __launch_bounds__(256)
transfer_tile_kernel(const int64_t* __restrict__ group_off, int max_runs, int64_t n_runs, int stat_stride,
                     const int64_t* __restrict__ a_row, const int32_t* __restrict__ a_fw,
                     const int64_t* __restrict__ a_xo, const double* __restrict__ ZA,
                     const int64_t* __restrict__ b_row, const int32_t* __restrict__ b_fw,
                     const int64_t* __restrict__ b_xo, const double* __restrict__ ZB, int ld,
                     double* __restrict__ out) {
    __shared__ double Si[kTT][kTS + 1], Su[kTT][kTS + 1];
    __shared__ int64_t xi[kTT], xu[kTT];
    const int q = blockIdx.x;
    int start[RS_MAXRUNS + 1], F = 0;
    const int N = rs_group_layout(q, group_off, max_runs, n_runs, a_row, a_fw, b_fw, stat_stride, start, F);
    if (N < 0 || N > ld) return;
    const int VB = (int)(b_row[q + 1] - b_row[q]);
    if (CROSS && (VB < 1 || VB > RS_MAXV)) return;
    const int rows = CROSS ? VB : N;
    const int tu_n = (N + kTT - 1) / kTT;
    int ti, tu;
    if constexpr (CROSS) {
        ti = (int)blockIdx.y / tu_n;
        tu = (int)blockIdx.y - ti * tu_n;
    } else {                                   // tile t = ti (ti + 1) / 2 + tu, tu <= ti
        ti = 0;
        while ((ti + 1) * (ti + 2) / 2 <= (int)blockIdx.y) ++ti;
        tu = (int)blockIdx.y - ti * (ti + 1) / 2;
    }
    const int i0 = ti * kTT, u0 = tu * kTT;
    if (i0 >= rows || u0 >= N) return;
    const int64_t g0 = group_off[q];
    const int tid = threadIdx.x;
    if (tid < 2 * kTT) {                       // element offsets of the tile's rows
        const int k = tid & (kTT - 1);
        const int v = (tid < kTT ? i0 : u0) + k;
        int64_t x = -1;
        if (tid < kTT && CROSS) {
            if (v < rows) x = b_xo[q] + (int64_t)v * F;
        } else if (v < N) {
            int r = 0;
            while (v >= start[r + 1]) ++r;
            x = a_xo[g0 + r] + (int64_t)(v - start[r]) * F;
        }
        (tid < kTT ? xi : xu)[k] = x;
    }
    __syncthreads();
    const double* Zi = CROSS ? ZB : ZA;
    const int tx = tid & 15, ty = tid >> 4;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int f0 = 0; f0 < F; f0 += kTS) {
        const int w = F - f0 < kTS ? F - f0 : kTS;
        for (int e = tid; e < 2 * kTT * kTS; e += 256) {   // lane c of warp-row r: feature f0 + c
            const int r = e / kTS, c = e - r * kTS;
            const bool isu = r >= kTT;
            const int rr = isu ? r - kTT : r;
            const int64_t x = isu ? xu[rr] : xi[rr];
            const double v = (x >= 0 && c < w) ? __ldg((isu ? ZA : Zi) + x + f0 + c) : 0.0;
            (isu ? Su : Si)[rr][c] = v;
        }
        __syncthreads();
        for (int c = 0; c < w; ++c) {
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const double zi = Si[ty + 16 * a][c];
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const double zu = Su[tx + 16 * b][c];
                    if constexpr (DIST) {
                        const double d = __dsub_rn(zi, zu);
                        acc[a][b] = __dadd_rn(acc[a][b], __dmul_rn(d, d));
                    } else {
                        acc[a][b] = fma(zi, zu, acc[a][b]);
                    }
                }
            }
        }
        __syncthreads();
    }
    const int64_t rows_ld = CROSS ? RS_MAXV : ld;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + ty + 16 * a, u = u0 + tx + 16 * b;
            if (i < rows && u < N && (CROSS || u <= i)) out[((int64_t)q * rows_ld + i) * ld + u] = acc[a][b];
        }
}

}  // namespace

cudaError_t rs_launch_transfer_blocks(const rs_batch* train_std, const rs_batch* test_std, const int64_t* group_off,
                                      int max_runs, int stat_stride, int ld, double* KA, double* Kx, int dist,
                                      cudaStream_t st) {
    const unsigned Q = (unsigned)test_std->n_programs;
    const int n = RS_MAXV * max_runs;
    const double* ZA = (const double*)train_std->X;
    const double* ZB = (const double*)test_std->X;
    const int nt = (n + kTT - 1) / kTT;        // tiles along the group's versions
    if (KA) {
        dim3 grid(Q, (unsigned)(nt * (nt + 1) / 2));
        transfer_tile_kernel<false, false><<<grid, 256, 0, st>>>(
            group_off, max_runs, train_std->n_programs, stat_stride, train_std->row_offsets, train_std->feat_width, train_std->x_offsets,
            ZA, test_std->row_offsets, test_std->feat_width, test_std->x_offsets, ZB, ld, KA);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    dim3 grid(Q, (unsigned)((RS_MAXV / kTT) * nt));
    if (dist) {
        dim3 g1(Q, (unsigned)(((int64_t)RS_MAXV * n + 127) / 128));
        transfer_block_kernel<true, true><<<g1, 128, 0, st>>>(
            group_off, max_runs, train_std->n_programs, stat_stride, train_std->row_offsets, train_std->feat_width, train_std->x_offsets,
            ZA, test_std->row_offsets, test_std->feat_width, test_std->x_offsets, ZB, ld, Kx);
    } else
        transfer_tile_kernel<true, false><<<grid, 256, 0, st>>>(
            group_off, max_runs, train_std->n_programs, stat_stride, train_std->row_offsets, train_std->feat_width, train_std->x_offsets,
            ZA, test_std->row_offsets, test_std->feat_width, test_std->x_offsets, ZB, ld, Kx);
    return cudaGetLastError();
}

#ifndef RS_GRAM_MAXB
#define RS_GRAM_MAXB 4
#endif
cudaError_t rs_launch_gram_f64(const rs_batch* b, double* K, int* dstatus, cudaStream_t st) {
    dim3 grid((unsigned)b->n_programs, kGramChunks);
    const size_t pad = rs_residency_pad(RS_GRAM_MAXB, sizeof(double) * 2 * RS_MAXV * kGramLd);
    if (pad) cudaFuncSetAttribute(gram_f64_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pad);
    gram_f64_kernel<false><<<grid, kGramThreads, pad, st>>>(b->n_programs, b->row_offsets, b->feat_width,
                                            b->x_offsets, (const double*)b->X, K, dstatus);
    return cudaGetLastError();
}

cudaError_t rs_launch_dist2_f64(const rs_batch* b, double* K, int* dstatus, cudaStream_t st) {
    dim3 grid((unsigned)b->n_programs, kGramChunks);
    gram_f64_kernel<true><<<grid, kGramThreads, 0, st>>>(b->n_programs, b->row_offsets, b->feat_width,
                                            b->x_offsets, (const double*)b->X, K, dstatus);
    return cudaGetLastError();
}
