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
//  - Set-up: the first call on each device looks up the array's device address with
//    cudaGetSymbolAddress while that device is current, and caches it.  Make that first
//    call before capturing any stream on that device.
//  - Sharing: all calls on a device use the same array and it keeps the previous call's
//    contents; each call clears the parts that must start at zero (LF-speed slots and the
//    status word) on its own stream.  Calls whose work overlaps on the GPU (different
//    streams without ordering between them) race on the array and give wrong results.
//  - Device-detected conditions (non-finite values, rho <= 0, p <= 0) are not reported by
//    this variant: its status word is cleared by the next call.
//
// No cudaMalloc, cudaFree or allocating library routine is called here.
#include <cstring>
#include <mutex>

#include "../../include/wenozn.h"
#include "launch.h"

using namespace wz;

namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_mutex;
void* g_scratch_dev[kMaxDevices] = {};

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" wenozn_status wenozn_rhs_noalloc(const wenozn_problem* p, const double* U, double* L,
                                            void* stream) {
    size_t unused = 0;
    wenozn_status st = wenozn_workspace_size(p, &unused);   // validates the problem
    if (st != WENOZN_OK) return st;
    if (!U || !L || U == L) return WENOZN_EINVAL;
    const size_t nv = p->system == WENOZN_ADVECTION_1D ? 1 : (p->system == WENOZN_EULER_1D ? 3 : 4);
    const size_t nx = size_t(p->nx), ny = size_t(p->ny);
    const size_t off_fx = align_up(sizeof(Ctrl));
    const size_t off_gy = off_fx + align_up(nv * (nx + 1) * ny * sizeof(double));
    const size_t need = off_gy + (p->system == WENOZN_EULER_2D ? align_up(nv * nx * (ny + 1) * sizeof(double)) : 0);
    if (need > kStaticScratchBytes) return WENOZN_ENOMEM_WS;

    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return WENOZN_ECUDA;
    char* b = static_cast<char*>(base);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(b);
    double* fx = reinterpret_cast<double*>(b + off_fx);
    double* gy = reinterpret_cast<double*>(b + off_gy);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    const bool per_field = p->split == WENOZN_SPLIT_LF_FIELD && p->system != WENOZN_ADVECTION_1D;
    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s);
    if (e == cudaSuccess)
        e = launch_max_wavespeed(p->system, U, int64_t(nx * ny), p->gamma, p->adv_speed, ctrl->alpha[0],
                                 &ctrl->status, s, per_field ? &ctrl->alpha_f[0][0][0] : nullptr);
    FluxArgs fa;
    fa.U = U;
    fa.after_x = 0;
    fa.alpha_bits = ctrl->alpha[0];
    fa.alpha_f_bits = &ctrl->alpha_f[0][0][0];
    fa.weights = p->weights;
    fa.split = p->split;
    fa.nx = p->nx;
    fa.ny = p->ny;
    fa.eps4 = 4.0 * p->eps;
    fa.kappa = zn_kappa(p->A);
    fa.fast_rcp = zn_fast_rcp(p->eps, p->A, p->weights);
    fa.gamma = p->gamma;
    fa.adv_speed = p->adv_speed;
    if (e == cudaSuccess) {
        fa.Fout = fx;
        fa.bc = p->bc_x;
        e = launch_flux(p->system, 0, fa, s);
    }
    if (e == cudaSuccess && p->system == WENOZN_EULER_2D) {
        fa.Fout = gy;
        fa.bc = p->bc_y;
        e = launch_flux(p->system, 1, fa, s);
    }
    if (e == cudaSuccess) {
        UpdateArgs u;
        std::memset(&u, 0, sizeof u);
        u.Fx = fx;
        u.Gy = gy;
        u.nx = p->nx;
        u.ny = p->ny;
        u.rdx = 1.0 / p->dx;
        u.rdy = p->system == WENOZN_EULER_2D ? 1.0 / p->dy : 0.0;
        u.mode = 0;
        u.out = L;
        u.ctrl = ctrl;
        u.next_slot = -1;
        u.clear_slot = -1;
        u.alpha_next = nullptr;
        u.field_speeds = 0;
        u.gamma = p->gamma;
        u.adv_speed = p->adv_speed;
        e = launch_update(p->system, u, s);
    }
    note_status(stream, &ctrl->status);
    return e == cudaSuccess ? WENOZN_OK : WENOZN_ECUDA;
}
