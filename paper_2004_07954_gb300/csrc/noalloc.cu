// wenozn_rhs_noalloc: the right-hand side of wenozn_rhs for callers that cannot allocate.
//
// Some callers have no way to hand the library a device workspace: code that runs where
// cudaMalloc is unavailable or forbidden (inside a host callback or a driver-managed
// plug-in that must not allocate, under a memory pool that is fully reserved, or in a
// process that may only use memory set aside when the module was loaded).  For them this
// variant takes its scratch (the 256-byte control block and the interface-flux buffers)
// from a fixed array in the library's own device memory instead of a workspace.
//
//  - Size: kStaticScratchBytes = 8 MiB.  Every GPU on which the library is loaded holds
//    this array until the process exits.  Problems whose scratch would not fit are
//    rejected with WENOZN_ENOMEM_WS before anything is enqueued (2D Euler up to about
//    131,000 cells, 1D Euler up to about 349,000 cells, advection up to about 1,048,000).
//  - Set-up: every call looks up the array's device address with cudaGetSymbolAddress
//    while the caller's device is current (a lookup, not an allocation), so the address is
//    never stale, even after a device reset.  The first call on a device also loads the
//    library's device code there; make it before capturing any stream on that device.
//  - Sharing: all calls on a device use the same array and it keeps the previous call's
//    contents; each call clears the parts that must start at zero (LF-speed slots and the
//    status word) on its own stream.  Calls whose work overlaps on the GPU (different
//    streams without ordering between them) race on the array and give wrong results.
//  - Device-detected conditions (non-finite values, rho <= 0, p <= 0) are not reported by
//    this variant: its status word lives in the shared array, is cleared by the next call
//    and is not registered with wenozn_last_error.
//
// No cudaMalloc, cudaFree or allocating library routine is called here.
#include "host_common.h"

using namespace wz;

namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

}  // namespace

extern "C" wenozn_status wenozn_rhs_noalloc(const wenozn_problem* p, const double* U, double* L,
                                            void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U || !L || U == L) return WENOZN_EINVAL;
    // the control block and the interface fluxes, laid out as in a workspace without the
    // two RK stage buffers
    const size_t nv = size_t(nvar_of(p->system));
    const size_t nx = size_t(p->nx), ny = size_t(p->ny);
    const size_t off_fx = align_up(sizeof(Ctrl));
    const size_t off_gy = off_fx + align_up(nv * (nx + 1) * ny * sizeof(double));
    const size_t need = off_gy + (p->system == WENOZN_EULER_2D ? align_up(nv * nx * (ny + 1) * sizeof(double)) : 0);
    if (need > kStaticScratchBytes) return WENOZN_ENOMEM_WS;

    // the array's address on the current device (host code may not use g_scratch itself)
    void* base = nullptr;
    if (cudaGetSymbolAddress(&base, g_scratch) != cudaSuccess || !base) return WENOZN_ECUDA;
    char* b = static_cast<char*>(base);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(b);
    double* fx = reinterpret_cast<double*>(b + off_fx);
    double* gy = reinterpret_cast<double*>(b + off_gy);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s);
    if (e == cudaSuccess)
        e = launch_max_wavespeed(p->system, U, int64_t(nx * ny), p->gamma, p->adv_speed, ctrl->alpha[0],
                                 &ctrl->status, s, field_slot(*p, ctrl, 0));
    if (e == cudaSuccess) e = launch_fluxes(*p, U, ctrl->alpha[0], &ctrl->alpha_f[0][0][0], fx, gy, s);
    if (e == cudaSuccess) {
        UpdateArgs u = update_args(*p, ctrl, fx, gy);
        u.mode = 0;
        u.out = L;
        e = launch_update(p->system, u, s);
    }
    return cuda_status(e);
}
