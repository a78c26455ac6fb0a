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
#ifdef __cplusplus
}
#endif
#endif
