// Diagnostics (include/wenozn_diag.h): the reciprocal check behind the reconstruction's
// f^ = c + num/den and the FP64 FMA rate probe.  Test and measurement aids only; the solver
// does not use this translation unit.
#include "../../include/wenozn_diag.h"
#include "launch.h"

using namespace wz;

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) rcp_check_kernel(const double* d, int64_t n, double* fast,
                                                              double* ieee) {
    const int64_t i = blockIdx.x * int64_t(kThreads) + threadIdx.x;
    if (i >= n) return;
    fast[i] = rcp_nr(d[i]);
    ieee[i] = 1.0 / d[i];
}

// FP64 FMA rate probe: four independent FMA chains per thread and no memory traffic in the
// loop; every thread stores its sum through a pointer argument (into a static buffer for up
// to kProbeBlocks blocks).  Measured on GB300: a conditional store, or a store to the
// device symbol itself, made the same loop run at 0.84 of this rate.
constexpr int kProbeBlocks = 512;
__device__ double g_fma_out[kProbeBlocks * kThreads];

__global__ void __launch_bounds__(kThreads) fma_probe_kernel(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1.0, x2 = x0 + 2.0, x3 = x0 + 3.0;
    for (int it = 0; it < iters; ++it) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
    }
    out[blockIdx.x * kThreads + threadIdx.x] = (x0 + x1) + (x2 + x3);
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 152;
    return sms > 0 ? sms : 152;
}

// Times sm_count x 2 blocks of 256 threads, each thread fmas_per_thread independent FP64
// FMAs (four chains), after one warm-up launch; writes the achieved GFLOP/s (2 per FMA).
cudaError_t measure_fma_rate(int64_t fmas_per_thread, double* gflops, cudaStream_t s) {
    const int grid = 2 * sm_count() < kProbeBlocks ? 2 * sm_count() : kProbeBlocks;
    const int iters = int(fmas_per_thread / 4);
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&out), g_fma_out);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        fma_probe_kernel<<<grid, kThreads, 0, s>>>(out, iters, 0.999999, 1e-7);     // warm-up
        e = cudaEventRecord(e0, s);
    }
    if (e == cudaSuccess) {
        fma_probe_kernel<<<grid, kThreads, 0, s>>>(out, iters, 0.999999, 1e-7);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) *gflops = ms > 0.0f ? 2.0 * 4.0 * double(iters) * grid * kThreads / (ms * 1e6) : 0.0;
    return e;
}

}  // namespace

extern "C" {

wenozn_status wenozn_check_reciprocal(const double* d, int64_t n, double* fast, double* ieee,
                                      void* stream) {
    if (!d || !fast || !ieee || n < 1 || n > (int64_t(1) << 31)) return WENOZN_EINVAL;
    rcp_check_kernel<<<unsigned((n + kThreads - 1) / kThreads), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        d, n, fast, ieee);
    return cudaGetLastError() == cudaSuccess ? WENOZN_OK : WENOZN_ECUDA;
}

wenozn_status wenozn_fp64_fma_rate(int64_t fmas_per_thread, double* gflops, void* stream) {
    if (!gflops || fmas_per_thread < 4 || fmas_per_thread > (int64_t(1) << 32)) return WENOZN_EINVAL;
    return measure_fma_rate(fmas_per_thread, gflops, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? WENOZN_OK : WENOZN_ECUDA;
}

}  // extern "C"
