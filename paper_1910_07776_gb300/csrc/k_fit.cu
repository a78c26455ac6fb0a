// K3 + K4: batched ridge fits, predictions, ranking and scoring (Sec. 2 tiers 2 and 3,
// Sec. 3.3 pairs, Sec. 3.4 regression family, Sec. 5 protocol, Sec. 6 / Table 3 metric).
//
// Work unit: a chunk of up to kChunk consecutive splits of one program.  A persistent grid
// pulls chunks from an atomic queue; the program's Gram block, masks, log times and pair
// lists are staged in shared memory once per program change.
//
// Fit (per split s and optimization j): the n training pairs are the pairs (v, v|j) with
// both versions in the train mask.  With the Gram block K (uncentred), the ridge problem
// with an unpenalised intercept is the bordered system
//       (K_TT + lambda I) alpha + b 1 = y,      1^T alpha = 0,
// (stationarity in beta = sum_a alpha_a z_a and in b).  With M = K_TT + lambda I = L L^T
// (FP64 Cholesky): u = M^-1 y, w = M^-1 1, b = 1^T u / 1^T w, alpha = u - b w; the
// prediction for a test version t is b + sum_a alpha_a K[t][v_a] = b + z_t . beta.
//
// The FP64 pipe of this part is narrow, so the kernel keeps its FP64 lanes busy:
//   - batched form: fits with n <= SMALL are solved one per thread; fits are sorted by n
//     (descending) so a warp's 32 fits have nearly the same size; each lane's packed
//     triangle lives in shared memory interleaved across lanes (conflict-free);
//   - larger fits (and every fit in the plain form) are solved one per warp, lanes = rows.
// Predict/rank: one thread per (split, test row): six dot products over the fit's pairs,
// an insertion sort of at most six keys, threshold, top-k, counters.
#include <math.h>

#include "rs_internal.cuh"

namespace {

constexpr int kChunk = 16;
constexpr int kFits = kChunk * RS_NOPT;
constexpr int kKld = RS_MAXV + 1;   // padded row stride of the Gram block in shared memory

__host__ __device__ constexpr int tri(int n) { return n * (n + 1) / 2; }

template <int WARPS, int SMALL>
struct FitSmem {
    static constexpr int kLaneNeed = tri(SMALL) + 2 * SMALL;         // L, 1/diag, w
    static constexpr int kPoolSmall = kLaneNeed * 32;
    static constexpr int kPoolLarge = 32 * 33;
    static constexpr int kPool = kPoolSmall > kPoolLarge ? kPoolSmall : kPoolLarge;
    double K[RS_MAXV * kKld];
    double lt[RS_MAXV];
    double ylab[RS_NOPT][RS_MAXPAIRS];
    double coef[kFits][RS_COEF_STRIDE];
    double pool[WARPS][kPool];
    uint64_t tmask[kChunk];
    uint32_t pmask[kFits];
    int row_base[kChunk + 1];
    int npair[RS_NOPT];
    int16_t small_list[kFits];
    int16_t large_list[kFits];
    uint8_t nfit[kFits];
    uint8_t status[kFits];
    uint8_t pair_b[RS_NOPT][RS_MAXPAIRS];
    uint8_t pair_a[RS_NOPT][RS_MAXPAIRS];
    uint8_t vidx[WARPS][32][RS_MAXPAIRS];
    uint8_t msk[RS_MAXV];
    int8_t slot_of[RS_MAXV];
    int n_small, n_large;
    int cur_prog, V, item, prog_ok;
};

// The a-th set bit (0-based) of x; x must have more than a set bits.
__device__ __forceinline__ int select_bit(uint64_t x, int a) {
    for (int i = 0; i < a; ++i) x &= x - 1;
    return __ffsll((long long)x) - 1;
}

// ------------------------------------------------------------------ one fit per thread
// Packed lower triangle L (row-major), reciprocal diagonal and w live at reg[e * 32].
// u (then alpha) lives in coef[1..n]; coef[0] receives b.
template <int SMALL>
__device__ int fit_thread(int n, const uint8_t* vlist, const double* K, double lambda,
                          double* reg, double* coef) {
    double* L = reg;
    double* rinv = reg + tri(SMALL) * 32;
    double* w = rinv + SMALL * 32;
    for (int i = 0; i < n; ++i) {
        const int vi = vlist[i];
        const int ti = tri(i);
        for (int k = 0; k <= i; ++k) {
            double s = K[vi * kKld + vlist[k]];
            if (k == i) s += lambda;
            const int tk = tri(k);
            for (int m = 0; m < k; ++m) s = fma(-L[(ti + m) * 32], L[(tk + m) * 32], s);
            if (k < i) {
                L[(ti + k) * 32] = s * rinv[k * 32];
            } else {
                if (!(s > 0.0)) return RS_FIT_NOTPD;
                const double d = sqrt(s);
                L[(ti + i) * 32] = d;
                rinv[i * 32] = 1.0 / d;
            }
        }
    }
    double* u = coef + 1;   // holds y on entry
    for (int i = 0; i < n; ++i) {
        const int ti = tri(i);
        double su = u[i], sw = 1.0;
        for (int k = 0; k < i; ++k) {
            const double l = L[(ti + k) * 32];
            su = fma(-l, u[k], su);
            sw = fma(-l, w[k * 32], sw);
        }
        u[i] = su * rinv[i * 32];
        w[i * 32] = sw * rinv[i * 32];
    }
    for (int i = n - 1; i >= 0; --i) {
        double su = u[i], sw = w[i * 32];
        for (int k = i + 1; k < n; ++k) {
            const double l = L[(tri(k) + i) * 32];
            su = fma(-l, u[k], su);
            sw = fma(-l, w[k * 32], sw);
        }
        u[i] = su * rinv[i * 32];
        w[i * 32] = sw * rinv[i * 32];
    }
    double su = 0.0, sw = 0.0;
    for (int i = 0; i < n; ++i) {
        su += u[i];
        sw += w[i * 32];
    }
    const double b = su / sw;
    bool finite = isfinite(b);
    for (int i = 0; i < n; ++i) {
        const double a = fma(-b, w[i * 32], u[i]);
        u[i] = a;
        finite = finite && isfinite(a);
    }
    coef[0] = b;
    return finite ? RS_FIT_OK : RS_FIT_NONFINITE;
}

// ------------------------------------------------------------------ one fit per warp
// Lane a owns row a (a < n <= 32).  Lsh: [32][33] doubles.  Returns a warp-uniform status.
__device__ int fit_warp(int n, uint32_t pm, const uint8_t* pair_b, const double* ylab,
                        const double* K, double lambda, double* Lsh, double* coef) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < n;
    int v = 0;
    double y = 0.0;
    if (act) {
        const int q = select_bit(pm, lane);
        v = pair_b[q];
        y = ylab[q];
    }
    double rinv = 0.0;
    for (int jj = 0; jj < n; ++jj) {
        const int vj = __shfl_sync(0xffffffffu, v, jj);
        double s = 0.0;
        if (act && lane >= jj) {
            s = K[v * kKld + vj];
            if (lane == jj) s += lambda;
            for (int m = 0; m < jj; ++m) s = fma(-Lsh[lane * 33 + m], Lsh[jj * 33 + m], s);
        }
        const double d = __shfl_sync(0xffffffffu, s, jj);
        if (!(d > 0.0)) return RS_FIT_NOTPD;
        const double ljj = sqrt(d);
        const double r = 1.0 / ljj;
        if (lane == jj) {
            Lsh[jj * 33 + jj] = ljj;
            rinv = r;
        } else if (act && lane > jj) {
            Lsh[lane * 33 + jj] = s * r;
        }
        __syncwarp();
    }
    double u = y, w = act ? 1.0 : 0.0;
    for (int kk = 0; kk < n; ++kk) {          // forward: L t = rhs
        const double r = __shfl_sync(0xffffffffu, rinv, kk);
        const double uk = __shfl_sync(0xffffffffu, u, kk) * r;
        const double wk = __shfl_sync(0xffffffffu, w, kk) * r;
        if (lane == kk) {
            u = uk;
            w = wk;
        } else if (act && lane > kk) {
            const double l = Lsh[lane * 33 + kk];
            u = fma(-l, uk, u);
            w = fma(-l, wk, w);
        }
    }
    for (int kk = n - 1; kk >= 0; --kk) {     // backward: L^T x = t
        const double r = __shfl_sync(0xffffffffu, rinv, kk);
        const double uk = __shfl_sync(0xffffffffu, u, kk) * r;
        const double wk = __shfl_sync(0xffffffffu, w, kk) * r;
        if (lane == kk) {
            u = uk;
            w = wk;
        } else if (lane < kk) {
            const double l = Lsh[kk * 33 + lane];
            u = fma(-l, uk, u);
            w = fma(-l, wk, w);
        }
    }
    double su = act ? u : 0.0, sw = act ? w : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        su += __shfl_xor_sync(0xffffffffu, su, o);
        sw += __shfl_xor_sync(0xffffffffu, sw, o);
    }
    const double b = su / sw;
    const double a = fma(-b, w, u);
    const int fin = __all_sync(0xffffffffu, !act || isfinite(a)) && isfinite(b);
    if (act) coef[1 + lane] = a;
    if (lane == 0) coef[0] = b;
    __syncwarp();
    return fin ? RS_FIT_OK : RS_FIT_NONFINITE;
}

template <int WARPS, int SMALL>
__global__ void __launch_bounds__(WARPS * 32, 1)
fit_predict_kernel(const rs_fit_args a) {
    using Sm = FitSmem<WARPS, SMALL>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm& sm = *reinterpret_cast<Sm*>(smem_raw);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NT = WARPS * 32;
    const int64_t n_items = (a.S + kChunk - 1) / kChunk;
    uint32_t cnt[RS_NCOUNTERS];
#pragma unroll
    for (int c = 0; c < RS_NCOUNTERS; ++c) cnt[c] = 0;
    const bool fit_in_launch = (a.coef_in == nullptr);
    const int NPLUS = RS_COEF_STRIDE;

    if (tid == 0) sm.cur_prog = -1;
    for (;;) {
        __syncthreads();
        if (tid == 0) sm.item = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        const int64_t item = sm.item;
        if (item >= n_items) break;
        int64_t s0 = item * kChunk;
        const int64_t s1 = min(s0 + (int64_t)kChunk, a.S);
        while (s0 < s1) {
            const int p = rs_find_segment(a.split_offsets, a.P, s0);
            const int64_t seg_end = min(s1, a.split_offsets[p + 1]);
            const int ns = (int)(seg_end - s0);
            // ---------------------------------------------------------- stage program p
            if (p != sm.cur_prog) {
                __syncthreads();
                const int64_t r0 = a.row_offsets[p];
                const int V = (int)(a.row_offsets[p + 1] - r0);
                const bool ok = V >= 1 && V <= RS_MAXV;
                if (!ok && tid == 0) rs_dev_flag(a.dstatus, RS_EDATA, p);
                if (ok) {
                    const double* Kg = a.K + (int64_t)p * RS_GRAM_LD * RS_GRAM_LD;
                    for (int e = tid; e < V * RS_MAXV; e += NT) {
                        const int r = e >> 6, c = e & 63;
                        sm.K[r * kKld + c] = (c < V) ? Kg[e] : 0.0;
                    }
                    for (int r = tid; r < RS_MAXV; r += NT) {
                        sm.slot_of[r] = -1;
                        if (r < V) {
                            sm.lt[r] = a.log_time[r0 + r];
                            sm.msk[r] = a.masks[r0 + r] & 63;
                        }
                    }
                }
                __syncthreads();
                if (ok && tid < V) sm.slot_of[sm.msk[tid]] = (int8_t)tid;
                __syncthreads();
                if (ok && tid < RS_NOPT) {
                    const int j = tid;
                    int np = 0;
                    for (int v = 0; v < V; ++v) {
                        const int m = sm.msk[v];
                        if ((m >> j) & 1) continue;
                        const int w = sm.slot_of[m | (1 << j)];
                        if (w < 0) continue;
                        sm.pair_b[j][np] = (uint8_t)v;
                        sm.pair_a[j][np] = (uint8_t)w;
                        sm.ylab[j][np] = sm.lt[v] - sm.lt[w];
                        ++np;
                    }
                    sm.npair[j] = np;
                }
                if (tid == 0) {
                    sm.cur_prog = p;
                    sm.V = V;
                    sm.prog_ok = ok;
                }
                __syncthreads();
            }
            const int V = sm.V;
            if (!sm.prog_ok) {
                s0 = seg_end;
                continue;
            }
            const uint64_t full = rs_full_mask(V);
            // ---------------------------------------------------------- per-fit pair masks
            for (int i = tid; i < ns; i += NT) sm.tmask[i] = a.train_masks[s0 + i] & full;
            __syncthreads();
            for (int f = tid; f < ns * RS_NOPT; f += NT) {
                const int i = f / RS_NOPT, j = f % RS_NOPT;
                const uint64_t T = sm.tmask[i];
                uint32_t pm = 0;
                for (int q = 0; q < sm.npair[j]; ++q)
                    if (((T >> sm.pair_b[j][q]) & 1) && ((T >> sm.pair_a[j][q]) & 1)) pm |= 1u << q;
                sm.pmask[f] = pm;
                sm.nfit[f] = (uint8_t)__popc(pm);
                if (fit_in_launch) {
                    // place the labels where the solver expects u
                    int aa = 0;
                    for (uint32_t x = pm; x; x &= x - 1) sm.coef[f][1 + aa++] = sm.ylab[j][__ffs(x) - 1];
                } else {
                    const double* src = a.coef_in + (s0 * RS_NOPT + f) * (int64_t)NPLUS;
                    for (int e = 0; e < NPLUS; ++e) sm.coef[f][e] = src[e];
                    sm.status[f] = isfinite(sm.coef[f][0]) ? RS_FIT_OK : RS_FIT_EMPTY;
                }
            }
            __syncthreads();
            if (fit_in_launch) {
                // ------------------------------------------------------ bin fits by size
                // Each fit computes its own position: small fits sorted by n descending
                // (ties by fit index), large fits in fit order.  Integer work only.
                {
                    const int nf = ns * RS_NOPT;
                    const bool plain = (a.form == RS_FORM_PLAIN);
                    int my_small = 0, my_large = 0;
                    for (int f = tid; f < kFits; f += NT) {
                        if (f >= nf) continue;
                        const int n = sm.nfit[f];
                        const bool is_large = n > 0 && (plain || n > SMALL);
                        const bool is_small = n > 0 && !is_large;
                        if (n == 0) {
                            sm.status[f] = RS_FIT_EMPTY;
                            sm.coef[f][0] = __longlong_as_double(0x7ff8000000000000ll);
                        }
                        int pos = 0;
                        for (int g = 0; g < nf; ++g) {
                            const int m = sm.nfit[g];
                            const bool gl = m > 0 && (plain || m > SMALL);
                            const bool gs = m > 0 && !gl;
                            if (is_small && gs && (m > n || (m == n && g < f))) ++pos;
                            if (is_large && gl && g < f) ++pos;
                        }
                        if (is_small) sm.small_list[pos] = (int16_t)f;
                        if (is_large) sm.large_list[pos] = (int16_t)f;
                        my_small += is_small;
                        my_large += is_large;
                    }
                    const int tot_small = __syncthreads_count(my_small);
                    const int tot_large = __syncthreads_count(my_large);
                    if (tid == 0) {
                        sm.n_small = tot_small;
                        sm.n_large = tot_large;
                    }
                }
                __syncthreads();
                // ------------------------------------------------------ small fits: one per lane
                const int groups = (sm.n_small + 31) / 32;
                for (int g = warp; g < groups; g += WARPS) {
                    const int e = g * 32 + lane;
                    if (e < sm.n_small) {
                        const int f = sm.small_list[e];
                        const int j = f % RS_NOPT;
                        const int n = sm.nfit[f];
                        uint8_t* vl = sm.vidx[warp][lane];
                        int aa = 0;
                        for (uint32_t x = sm.pmask[f]; x; x &= x - 1) vl[aa++] = sm.pair_b[j][__ffs(x) - 1];
                        sm.status[f] = (uint8_t)fit_thread<SMALL>(n, vl, sm.K, a.lambda,
                                                                 sm.pool[warp] + lane, sm.coef[f]);
                    }
                    __syncwarp();
                }
                // ------------------------------------------------------ large fits: one per warp
                for (int e = warp; e < sm.n_large; e += WARPS) {
                    const int f = sm.large_list[e];
                    const int j = f % RS_NOPT;
                    const int st = fit_warp(sm.nfit[f], sm.pmask[f], sm.pair_b[j], sm.ylab[j], sm.K,
                                            a.lambda, sm.pool[warp], sm.coef[f]);
                    if (lane == 0) sm.status[f] = (uint8_t)st;
                    __syncwarp();
                }
                __syncthreads();
                for (int f = tid; f < ns * RS_NOPT; f += NT) {
                    const int st = sm.status[f];
                    cnt[9] += st == RS_FIT_OK;
                    cnt[10] += st == RS_FIT_EMPTY;
                    cnt[11] += st == RS_FIT_NOTPD;
                    cnt[12] += st == RS_FIT_NONFINITE;
                    if (st != RS_FIT_OK) sm.coef[f][0] = __longlong_as_double(0x7ff8000000000000ll);
                }
                __syncthreads();
            }
            // ---------------------------------------------------------- fit outputs
            if (a.coef_out) {
                double* dst = a.coef_out + s0 * RS_NOPT * (int64_t)NPLUS;
                for (int e = tid; e < ns * RS_NOPT * NPLUS; e += NT) {
                    const int f = e / NPLUS, c = e % NPLUS;
                    const bool ok = sm.status[f] == RS_FIT_OK;
                    double v = sm.coef[f][c];
                    if (c > 0 && (!ok || c > sm.nfit[f])) v = 0.0;
                    dst[e] = v;
                }
            }
            if (a.status_out)
                for (int f = tid; f < ns * RS_NOPT; f += NT) a.status_out[s0 * RS_NOPT + f] = sm.status[f];
            // ---------------------------------------------------------- predict, rank, score
            if (a.rec_code) {
                if (tid == 0) {
                    int acc = 0;
                    for (int i = 0; i < ns; ++i) {
                        sm.row_base[i] = acc;
                        acc += V - __popcll(sm.tmask[i]);
                    }
                    sm.row_base[ns] = acc;
                }
                __syncthreads();
                const int R = sm.row_base[ns];
                for (int r = tid; r < R; r += NT) {
                    int i = 0;
                    while (sm.row_base[i + 1] <= r) ++i;
                    const int kth = r - sm.row_base[i];
                    const int t = select_bit(~sm.tmask[i] & full, kth);
                    const int64_t grow = a.rec_offsets[s0 + i] + kth;
                    const int mt = sm.msk[t];
                    double pred[RS_NOPT], act[RS_NOPT];
                    bool valid[RS_NOPT], known[RS_NOPT];
#pragma unroll
                    for (int j = 0; j < RS_NOPT; ++j) {
                        valid[j] = known[j] = false;
                        pred[j] = act[j] = __longlong_as_double(0x7ff8000000000000ll);
                        const bool has = (mt >> j) & 1;
                        if (has && !(a.flags & RS_RANK_ALL)) continue;
                        const int f = i * RS_NOPT + j;
                        if (sm.status[f] != RS_FIT_OK) {
                            cnt[13] += 1;
                            continue;
                        }
                        const double* cf = sm.coef[f];
                        double yh = cf[0];
                        int aa = 1;
                        for (uint32_t x = sm.pmask[f]; x; x &= x - 1)
                            yh = fma(cf[aa++], sm.K[t * kKld + sm.pair_b[j][__ffs(x) - 1]], yh);
                        pred[j] = yh;
                        valid[j] = true;
                        cnt[1] += 1;
                        if (!has) {
                            const int w = sm.slot_of[mt | (1 << j)];
                            if (w >= 0) {
                                act[j] = sm.lt[t] - sm.lt[w];
                                known[j] = true;
                                cnt[2] += 1;
                                if ((yh > 0.0) == (act[j] > 0.0)) cnt[3] += 1;
                            }
                        }
                    }
                    // insertion sort, descending; a later entry passes only if strictly larger
                    int order[RS_NOPT];
                    int m = 0;
#pragma unroll
                    for (int j = 0; j < RS_NOPT; ++j)
                        if (valid[j]) order[m++] = j;
                    for (int x = 1; x < m; ++x) {
                        const int cur = order[x];
                        int y = x - 1;
                        while (y >= 0 && pred[order[y]] < pred[cur]) {
                            order[y + 1] = order[y];
                            --y;
                        }
                        order[y + 1] = cur;
                    }
                    int c = 0;
                    int idx[RS_NOPT];
                    for (int x = 0; x < m && c < a.k; ++x)
                        if (pred[order[x]] >= a.log_tau) idx[c++] = order[x];
                    uint32_t code = (uint32_t)c;
                    for (int x = 0; x < RS_NOPT; ++x) code |= (uint32_t)(x < c ? idx[x] : 0xF) << (4 + 4 * x);
                    a.rec_code[grow] = code;
                    if (a.rec_pred)
                        for (int x = 0; x < a.k; ++x)
                            a.rec_pred[grow * a.k + x] = x < c ? pred[idx[x]] : __longlong_as_double(0x7ff8000000000000ll);
                    if (a.pred_all)
#pragma unroll
                        for (int j = 0; j < RS_NOPT; ++j) a.pred_all[grow * RS_NOPT + j] = pred[j];
                    cnt[0] += 1;
                    cnt[4] += c;
                    for (int x = 0; x < c; ++x)
                        if (known[idx[x]]) {
                            cnt[5] += 1;
                            if (act[idx[x]] > 0.0) cnt[6] += 1;
                        }
                    int bp = -1, ba = -1;
#pragma unroll
                    for (int j = 0; j < RS_NOPT; ++j) {
                        if (!(valid[j] && known[j])) continue;
                        if (bp < 0 || pred[j] > pred[bp]) bp = j;
                        if (ba < 0 || act[j] > act[ba]) ba = j;
                    }
                    if (bp >= 0) {
                        cnt[7] += 1;
                        if (bp == ba) cnt[8] += 1;
                    }
                }
            }
            __syncthreads();
            s0 = seg_end;
        }
    }
    if (a.counters) {
#pragma unroll
        for (int c = 0; c < RS_NCOUNTERS; ++c) {
            const uint32_t v = __reduce_add_sync(0xffffffffu, cnt[c]);
            if (lane == 0 && v) atomicAdd(a.counters + c, (unsigned long long)v);
        }
    }
}

template <int WARPS, int SMALL>
cudaError_t launch_fp(const rs_fit_args& a, cudaStream_t st) {
    using Sm = FitSmem<WARPS, SMALL>;
    auto kern = fit_predict_kernel<WARPS, SMALL>;
    const size_t smem = sizeof(Sm);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t items = (a.S + kChunk - 1) / kChunk;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > items) grid = items;
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(a.queue, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, WARPS * 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t rs_launch_fit_predict(const rs_fit_args& a, cudaStream_t st) {
    if (a.S == 0) return cudaSuccess;
    return launch_fp<4, 15>(a, st);
}
