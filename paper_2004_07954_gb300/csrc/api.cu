// C ABI of libwenozn.so: argument checks, workspace layout and the launch sequences of
// the RHS evaluation and the SSP-RK3 step.  Declarations and contracts: include/wenozn.h.
#include <cmath>
#include <cstring>

#include "../../include/wenozn.h"
#include "launch.h"

using namespace wz;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int nvar_of(int system) { return system == WENOZN_ADVECTION_1D ? 1 : (system == WENOZN_EULER_1D ? 3 : 4); }

struct Layout {
    size_t ctrl, u1, u2, fx, gy, total;
};

Layout layout_of(const wenozn_problem& p) {
    const size_t nv = size_t(nvar_of(p.system));
    const size_t nx = size_t(p.nx), ny = size_t(p.ny);
    Layout L;
    L.ctrl = 0;
    L.u1 = align_up(sizeof(Ctrl));
    L.u2 = L.u1 + align_up(nv * nx * ny * sizeof(double));
    L.fx = L.u2 + align_up(nv * nx * ny * sizeof(double));
    L.gy = L.fx + align_up(nv * (nx + 1) * ny * sizeof(double));
    L.total = L.gy + (p.system == WENOZN_EULER_2D ? align_up(nv * nx * (ny + 1) * sizeof(double)) : 0);
    return L;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

wenozn_status check_problem(const wenozn_problem* p) {
    if (!p) return WENOZN_EINVAL;
    if (p->system < 0 || p->system > 2 || p->flags != 0) return WENOZN_EINVAL;
    const bool two_d = p->system == WENOZN_EULER_2D;
    if (p->nx < 1 || p->nx > (1 << 30)) return WENOZN_EINVAL;
    if (two_d ? (p->ny < 1 || p->ny > (1 << 30)) : p->ny != 1) return WENOZN_EINVAL;
    if (int64_t(p->nx) * p->ny > (int64_t(1) << 34)) return WENOZN_EINVAL;
    if ((p->bc_x != WENOZN_BC_PERIODIC && p->bc_x != WENOZN_BC_OUTFLOW)) return WENOZN_EINVAL;
    if (two_d && p->bc_y != WENOZN_BC_PERIODIC && p->bc_y != WENOZN_BC_OUTFLOW) return WENOZN_EINVAL;
    if (!finite_pos(p->dx) || (two_d && !finite_pos(p->dy))) return WENOZN_EINVAL;
    if (!finite_pos(p->eps) || !std::isfinite(p->A) || p->A < 0.0 || !finite_pos(p->cfl)) return WENOZN_EINVAL;
    if (p->system == WENOZN_ADVECTION_1D) {
        if (!std::isfinite(p->adv_speed) || p->adv_speed == 0.0) return WENOZN_EINVAL;
    } else if (!std::isfinite(p->gamma) || p->gamma <= 1.0) {
        return WENOZN_EINVAL;
    }
    return WENOZN_OK;
}

wenozn_status cuda_status(cudaError_t e) { return e == cudaSuccess ? WENOZN_OK : WENOZN_ECUDA; }

// Launches the x (and y) flux kernels for stage input U with LF speeds in `alpha_bits`.
cudaError_t launch_fluxes(const wenozn_problem& p, const double* U, const unsigned long long* alpha_bits,
                          double* fx, double* gy, cudaStream_t s) {
    FluxArgs fa;
    fa.U = U;
    fa.alpha_bits = alpha_bits;
    fa.nx = p.nx;
    fa.ny = p.ny;
    fa.eps4 = 4.0 * p.eps;
    fa.A4 = 0.25 * p.A;
    fa.fast_rcp = zn_fast_rcp(p.eps, p.A);
    fa.gamma = p.gamma;
    fa.adv_speed = p.adv_speed;
    fa.Fout = fx;
    fa.bc = p.bc_x;
    cudaError_t e = launch_flux(p.system, 0, fa, s);
    if (e != cudaSuccess || p.system != WENOZN_EULER_2D) return e;
    fa.Fout = gy;
    fa.bc = p.bc_y;
    return launch_flux(p.system, 1, fa, s);
}

UpdateArgs update_args(const wenozn_problem& p, Ctrl* ctrl, const double* fx, const double* gy) {
    UpdateArgs u;
    std::memset(&u, 0, sizeof u);
    u.Fx = fx;
    u.Gy = gy;
    u.nx = p.nx;
    u.ny = p.ny;
    u.rdx = 1.0 / p.dx;
    u.rdy = p.system == WENOZN_EULER_2D ? 1.0 / p.dy : 0.0;
    u.ctrl = ctrl;
    u.next_slot = -1;
    u.cfl = p.cfl;
    u.dx = p.dx;
    u.dy = p.dy;
    u.gamma = p.gamma;
    u.adv_speed = p.adv_speed;
    return u;
}

char* ws_base(void* ws) { return static_cast<char*>(ws); }

}  // namespace

extern "C" {

wenozn_status wenozn_problem_init(wenozn_problem* p, int32_t system, int32_t nx, int32_t ny,
                                  double dx, double dy) {
    if (!p || system < 0 || system > 2) return WENOZN_EINVAL;
    std::memset(p, 0, sizeof *p);
    p->system = system;
    p->nx = nx;
    p->ny = system == WENOZN_EULER_2D ? ny : 1;
    p->bc_x = WENOZN_BC_OUTFLOW;
    p->bc_y = WENOZN_BC_OUTFLOW;
    p->dx = dx;
    p->dy = system == WENOZN_EULER_2D ? dy : 1.0;
    p->gamma = 1.4;
    p->eps = 1e-40;
    p->A = 10.0;
    p->cfl = 0.5;
    p->adv_speed = 1.0;
    return WENOZN_OK;
}

wenozn_status wenozn_workspace_size(const wenozn_problem* p, size_t* bytes) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!bytes) return WENOZN_EINVAL;
    *bytes = layout_of(*p).total;
    return WENOZN_OK;
}

wenozn_status wenozn_fill_ghosts(const wenozn_problem* p, double* U_padded, void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U_padded) return WENOZN_EINVAL;
    return cuda_status(launch_fill_ghosts(nvar_of(p->system), p->nx, p->ny, p->bc_x, p->bc_y,
                                          p->system == WENOZN_EULER_2D, U_padded,
                                          static_cast<cudaStream_t>(stream)));
}

wenozn_status wenozn_reconstruct(const double* f_padded, int64_t n, double* fhat, int32_t side,
                                 double eps, double A, void* stream) {
    if (!f_padded || !fhat || n < 1 || n > (int64_t(1) << 31) - 8) return WENOZN_EINVAL;
    if (side != 1 && side != -1) return WENOZN_EINVAL;
    if (!finite_pos(eps) || !std::isfinite(A) || A < 0.0) return WENOZN_EINVAL;
    return cuda_status(launch_reconstruct(f_padded, n, fhat, side, eps, A,
                                          static_cast<cudaStream_t>(stream)));
}

wenozn_status wenozn_max_wavespeed(const wenozn_problem* p, const double* U, double* alpha_out,
                                   int32_t* status_dev, void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U || !alpha_out) return WENOZN_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(alpha_out, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return WENOZN_ECUDA;
    return cuda_status(launch_max_wavespeed(p->system, U, int64_t(p->nx) * p->ny, p->gamma,
                                            p->adv_speed,
                                            reinterpret_cast<unsigned long long*>(alpha_out),
                                            status_dev, s));
}

wenozn_status wenozn_flux(const wenozn_problem* p, const double* U, const double* alpha,
                          int32_t dir, double* Fout, void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U || !Fout || U == Fout || (p->system != WENOZN_ADVECTION_1D && !alpha)) return WENOZN_EINVAL;
    if (dir != 0 && !(dir == 1 && p->system == WENOZN_EULER_2D)) return WENOZN_EINVAL;
    FluxArgs fa;
    fa.U = U;
    fa.alpha_bits = reinterpret_cast<const unsigned long long*>(alpha);
    fa.nx = p->nx;
    fa.ny = p->ny;
    fa.eps4 = 4.0 * p->eps;
    fa.A4 = 0.25 * p->A;
    fa.fast_rcp = zn_fast_rcp(p->eps, p->A);
    fa.gamma = p->gamma;
    fa.adv_speed = p->adv_speed;
    fa.Fout = Fout;
    fa.bc = dir == 0 ? p->bc_x : p->bc_y;
    return cuda_status(launch_flux(p->system, dir, fa, static_cast<cudaStream_t>(stream)));
}

wenozn_status wenozn_rhs(const wenozn_problem* p, const double* U, double* L, void* ws,
                         size_t ws_bytes, void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U || !L || !ws || U == L) return WENOZN_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return WENOZN_EINVAL;
    const Layout lay = layout_of(*p);
    if (ws_bytes < lay.total) return WENOZN_ENOMEM_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws_base(ws) + lay.ctrl);
    double* fx = reinterpret_cast<double*>(ws_base(ws) + lay.fx);
    double* gy = reinterpret_cast<double*>(ws_base(ws) + lay.gy);
    cudaError_t e = cudaMemsetAsync(ctrl->alpha, 0, sizeof(ctrl->alpha), s);
    if (e == cudaSuccess)
        e = launch_max_wavespeed(p->system, U, int64_t(p->nx) * p->ny, p->gamma, p->adv_speed,
                                 ctrl->alpha[0], &ctrl->status, s);
    if (e == cudaSuccess) e = launch_fluxes(*p, U, ctrl->alpha[0], fx, gy, s);
    if (e == cudaSuccess) {
        UpdateArgs u = update_args(*p, ctrl, fx, gy);
        u.mode = 0;
        u.out = L;
        e = launch_update(p->system, u, s);
    }
    return cuda_status(e);
}

wenozn_status wenozn_rk3_step(const wenozn_problem* p, double* U, double dt, double t_remaining,
                              double* dt_out, void* ws, size_t ws_bytes, void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U || !ws || std::isnan(dt) || std::isnan(t_remaining) || std::isinf(dt)) return WENOZN_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return WENOZN_EINVAL;
    const Layout lay = layout_of(*p);
    if (ws_bytes < lay.total) return WENOZN_ENOMEM_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws_base(ws) + lay.ctrl);
    double* u1 = reinterpret_cast<double*>(ws_base(ws) + lay.u1);
    double* u2 = reinterpret_cast<double*>(ws_base(ws) + lay.u2);
    double* fx = reinterpret_cast<double*>(ws_base(ws) + lay.fx);
    double* gy = reinterpret_cast<double*>(ws_base(ws) + lay.gy);
    const bool euler = p->system != WENOZN_ADVECTION_1D;

    cudaError_t e = cudaMemsetAsync(ctrl->alpha, 0, sizeof(ctrl->alpha), s);
    if (e == cudaSuccess)
        e = launch_max_wavespeed(p->system, U, int64_t(p->nx) * p->ny, p->gamma, p->adv_speed,
                                 ctrl->alpha[0], &ctrl->status, s);
    const double* stage_in[3] = {U, u1, u2};
    double* stage_out[3] = {u1, u2, U};
    for (int stage = 0; stage < 3 && e == cudaSuccess; ++stage) {
        e = launch_fluxes(*p, stage_in[stage], ctrl->alpha[stage], fx, gy, s);
        if (e != cudaSuccess) break;
        UpdateArgs u = update_args(*p, ctrl, fx, gy);
        u.mode = stage + 1;
        u.Us = stage_in[stage];
        u.Un = U;
        u.out = stage_out[stage];
        u.next_slot = (euler && stage < 2) ? stage + 1 : -1;
        u.dt_fixed = dt;
        u.t_remaining = t_remaining;
        e = launch_update(p->system, u, s);
    }
    if (e != cudaSuccess) return WENOZN_ECUDA;
    if (dt_out) {
        e = cudaMemcpyAsync(dt_out, &ctrl->dt, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return WENOZN_ECUDA;
    }
    return WENOZN_OK;
}

const double* wenozn_workspace_dt(const void* ws) {
    return ws ? &reinterpret_cast<const Ctrl*>(ws)->dt : nullptr;
}

wenozn_status wenozn_workspace_status(void* ws, int32_t* status, int32_t clear, void* stream) {
    if (!ws || !status) return WENOZN_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws);
    int32_t host = 0;
    cudaError_t e = cudaMemcpyAsync(&host, &ctrl->status, sizeof host, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && clear) e = cudaMemsetAsync(&ctrl->status, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return WENOZN_ECUDA;
    *status = host;
    return WENOZN_OK;
}

wenozn_status wenozn_check_reciprocal(const double* d, int64_t n, double* fast, double* ieee,
                                      void* stream) {
    if (!d || !fast || !ieee || n < 1 || n > (int64_t(1) << 31)) return WENOZN_EINVAL;
    return cuda_status(launch_rcp_check(d, n, fast, ieee, static_cast<cudaStream_t>(stream)));
}

const char* wenozn_status_string(wenozn_status s) {
    switch (s) {
        case WENOZN_OK: return "ok";
        case WENOZN_EINVAL: return "invalid argument";
        case WENOZN_ECUDA: return "CUDA launch or copy failed";
        case WENOZN_ENOMEM_WS: return "workspace too small";
        case WENOZN_ENONFINITE: return "non-finite value or non-positive density/pressure";
        case WENOZN_ETIMEOUT: return "bounded device-side wait gave up";
    }
    return "unknown status";
}

const char* wenozn_version(void) { return "0.1.0"; }

}  // extern "C"
