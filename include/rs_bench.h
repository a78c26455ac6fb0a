/*
 * rs_bench.h -- measurement helper of the rs library (not a step of the method; the paper
 * has no counterpart).  Used to state the arithmetic roofline of the FP64-bound kernels.
 */
#ifndef RS_BENCH_H_
#define RS_BENCH_H_
#include "rs.h"
#ifdef __cplusplus
extern "C" {
#endif
/* Runs independent fused multiply-add chains in 8 x 256-thread blocks per SM on the
 * current device (legacy default stream), `iters` iterations of 8 chains per thread,
 * and writes the best of three timed runs to *gflops (2 flops per FMA).  use_f64: 1 for
 * double, 0 for float.  Blocking; allocates and frees a few KiB.  RS_EINVAL for a NULL
 * output or iters < 1, RS_ECUDA if a CUDA call fails.                                  */
rs_status rs_measure_fma_peak(int use_f64, int iters, double* gflops);
/* Check of the solvers' FP64 reciprocal and reciprocal square root (an FP32 seed refined by
 * Newton / series steps, used for the pivots of the LDL^T and Cholesky factorisations of
 * Sec. 3.4's regression) against CUDA's correctly rounded division and square root: for
 * each of the n positive doubles d (device memory), out[4 i .. 4 i + 3] (device memory,
 * 4 n doubles, caller-owned) receives rcp(d_i), 1.0 / d_i, rsqrt(d_i) and 1.0 / sqrt(d_i).
 * Asynchronous on cuda_stream (NULL: the legacy default stream).  RS_EINVAL for n < 0 or a
 * NULL pointer with n > 0, RS_ECUDA if the launch fails.                               */
rs_status rs_check_reciprocals(const double* d, int64_t n, double* out, void* cuda_stream);
/* Check of the bounded waits of the asynchronous pipelines (the rank pass's TMA ring and the
 * tensor-core GEMM): one thread waits, through the same wait routine those kernels use, on
 * an mbarrier that nothing arrives at and no copy targets, with a limit of limit_ns
 * (1 us .. 100 ms) instead of their 1 s.  The wait gives up, the kernel sets RS_ETIMEOUT
 * (detail 99) in device_status[0..1] (device ints, caller-owned, to be zeroed by the
 * caller) and writes 0 to *completed (device int; 1 would mean the wait completed), and
 * returns; the context stays usable.  Asynchronous on cuda_stream.  RS_EINVAL for NULL
 * pointers or a limit out of range, RS_ECUDA if the launch fails.                     */
rs_status rs_check_wait_timeout(int* device_status, int* completed, int64_t limit_ns, void* cuda_stream);
#ifdef __cplusplus
}
#endif
#endif
