// Arithmetic-peak measurement used to state the ALU roofline of the FP64-bound kernels:
// independent FMA chains in every thread of a full grid, timed with CUDA events.  Also the
// device-side check of the solvers' reciprocal and reciprocal square root against CUDA's
// correctly rounded division and square root.
#include "mbar.cuh"
#include "rank_row.cuh"
#include "rs_internal.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x, x1 = x0 + (T)1, x2 = x0 + (T)2, x3 = x0 + (T)3;
    T x4 = x0 + (T)4, x5 = x0 + (T)5, x6 = x0 + (T)6, x7 = x0 + (T)7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == (T)-12345) out[blockIdx.x] = s;   // keeps the chains alive
}

// out[4 i .. 4 i + 3] = rcp_newton(d_i), 1.0 / d_i, rsqrt_newton(d_i), 1.0 / sqrt(d_i).
__global__ void __launch_bounds__(256) reciprocal_check_kernel(const double* __restrict__ d, int64_t n,
                                                               double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = d[i];
        out[4 * i + 0] = rcp_newton(x);
        out[4 * i + 1] = 1.0 / x;
        out[4 * i + 2] = rsqrt_newton(x);
        out[4 * i + 3] = 1.0 / sqrt(x);
    }
}

// One thread waits, with the kernels' bounded wait, on an mbarrier that nothing arrives at
// and no copy targets; after limit_ns the wait gives up, flags RS_ETIMEOUT (site 99) in the
// status word, and the kernel returns.  out[0] = 1 if the wait completed, 0 if it gave up.
__global__ void wait_timeout_kernel(int* dstatus, int* out, unsigned long long limit_ns) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x != 0) return;
    const uint32_t b = tc::smem_u32(&bar);
    tc::mbar_init(b, 1);
    tc::fence_barrier_init();
    out[0] = tc::mbar_wait_for(b, 0, dstatus, 99, limit_ns) ? 1 : 0;
}

}  // namespace

extern "C" rs_status rs_check_wait_timeout(int* device_status, int* completed, int64_t limit_ns,
                                           void* cuda_stream) {
    if (!device_status || !completed || limit_ns < 1000 || limit_ns > 100000000) return RS_EINVAL;
    wait_timeout_kernel<<<1, 32, 0, (cudaStream_t)cuda_stream>>>(device_status, completed,
                                                                 (unsigned long long)limit_ns);
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ECUDA;
}

extern "C" rs_status rs_check_reciprocals(const double* d, int64_t n, double* out, void* cuda_stream) {
    if (n < 0 || (n > 0 && (!d || !out))) return RS_EINVAL;
    if (n == 0) return RS_OK;
    const int64_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    reciprocal_check_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)cuda_stream>>>(d, n, out);
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ECUDA;
}

extern "C" rs_status rs_measure_fma_peak(int use_f64, int iters, double* gflops) {
    if (!gflops || iters < 1) return RS_EINVAL;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    void* out = nullptr;
    if (cudaMalloc(&out, blocks * sizeof(double)) != cudaSuccess) return RS_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0);
        if (use_f64) fma_chains<double><<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-7);
        else fma_chains<float><<<blocks, threads>>>((float*)out, iters, 0.999999f, 1e-7f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return RS_ECUDA;
    *gflops = 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e9;
    return RS_OK;
}
