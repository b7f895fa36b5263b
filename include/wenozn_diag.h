/*
 * wenozn_diag.h - diagnostics of libwenozn.so: measurement and test aids, not part of the
 * solver.  They check the arithmetic the solver relies on and measure the hardware it runs
 * on; nothing in wenozn.h calls them, and a user of the solver never needs them.
 *
 * Conventions as in wenozn.h (device/host pointers, `stream` a cudaStream_t as void*,
 * WENOZN_EINVAL for bad arguments before any CUDA call, WENOZN_ECUDA for CUDA failures).
 */
#ifndef WENOZN_DIAG_H
#define WENOZN_DIAG_H

#include "wenozn.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Test aid: evaluates, for n positive normal doubles d, the reciprocal the reconstruction
 * uses for f^ = c + num/den (the hardware approximation refined by one third-order
 * Householder step) into `fast`, and CUDA's IEEE 1/d into `ieee`, so that a test can bound
 * the former's error.
 *   d, fast, ieee : device, n doubles (1 <= n <= 2^31). */
wenozn_status wenozn_check_reciprocal(const double* d, int64_t n, double* fast, double* ieee,
                                      void* stream);

/* Measurement: the FP64 FMA rate this GPU sustains on pure register arithmetic (two blocks
 * of 256 threads per SM, four independent FMA chains per thread, fmas_per_thread FMAs each,
 * no memory traffic), timed with CUDA events on `stream` after one warm-up launch; the
 * call synchronizes `stream`.  Writes GFLOP/s (2 flops per FMA) to the host double
 * *gflops.  It is the achievable ceiling beside the nominal peak (2 FP64 FMA lanes per SM
 * per clock) against which the solver's FP64-bound kernels are measured.
 * EINVAL unless 4 <= fmas_per_thread <= 2^32 and gflops is non-NULL. */
wenozn_status wenozn_fp64_fma_rate(int64_t fmas_per_thread, double* gflops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* WENOZN_DIAG_H */
