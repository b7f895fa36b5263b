// Host-side helpers shared by the C-ABI translation units: argument checks and the layout
// of the caller's workspace.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>

#include "../../include/wenozn.h"
#include "launch.h"

namespace wz {

constexpr size_t kAlign = 256;

inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

inline int nvar_of(int system) { return system == WENOZN_ADVECTION_1D ? 1 : (system == WENOZN_EULER_1D ? 3 : 4); }

// Workspace regions of wenozn_rhs / wenozn_rk3_step, followed by the extra regions the
// adjoint entry points use (per-interface cotangent contributions for advection or the
// Euler stage kernel's correction records, their control words and two cotangent vectors).
struct Layout {
    size_t ctrl, u1, u2, fx, gy, total;        // forward
    size_t C, vjp_ctl, ub2, ub1, total_vjp;    // adjoint (1D only)
};

inline Layout layout_of(const wenozn_problem& p) {
    const size_t nv = size_t(nvar_of(p.system));
    const size_t nx = size_t(p.nx), ny = size_t(p.ny);
    Layout L;
    L.ctrl = 0;
    L.u1 = align_up(sizeof(Ctrl));
    L.u2 = L.u1 + align_up(nv * nx * ny * sizeof(double));
    L.fx = L.u2 + align_up(nv * nx * ny * sizeof(double));
    L.gy = L.fx + align_up(nv * (nx + 1) * ny * sizeof(double));
    L.total = L.gy + (p.system == WENOZN_EULER_2D ? align_up(nv * nx * (ny + 1) * sizeof(double)) : 0);
    L.C = L.total;
    L.vjp_ctl = L.C + align_up(vjp_contrib_doubles(int(nv), int(nx)) * sizeof(double));
    L.ub2 = L.vjp_ctl + kAlign;
    L.ub1 = L.ub2 + align_up(nv * nx * sizeof(double));
    L.total_vjp = L.ub1 + align_up(nv * nx * sizeof(double));
    return L;
}

inline bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

inline wenozn_status check_problem(const wenozn_problem* p) {
    if (!p) return WENOZN_EINVAL;
    if (p->system < 0 || p->system > 2 || p->flags != 0) return WENOZN_EINVAL;
    if (p->weights < 0 || p->weights > 3 || p->split < 0 || p->split > 3) return WENOZN_EINVAL;
    const bool two_d = p->system == WENOZN_EULER_2D;
    if (p->nx < 1 || p->nx > (1 << 30)) return WENOZN_EINVAL;
    if (two_d ? (p->ny < 1 || p->ny > (1 << 30)) : p->ny != 1) return WENOZN_EINVAL;
    if (int64_t(p->nx) * p->ny > (int64_t(1) << 34)) return WENOZN_EINVAL;
    if (p->bc_x < WENOZN_BC_PERIODIC || p->bc_x > WENOZN_BC_REFLECTIVE) return WENOZN_EINVAL;
    if (two_d && (p->bc_y < WENOZN_BC_PERIODIC || p->bc_y > WENOZN_BC_REFLECTIVE)) return WENOZN_EINVAL;
    if (!finite_pos(p->dx) || (two_d && !finite_pos(p->dy))) return WENOZN_EINVAL;
    if (!finite_pos(p->eps) || !finite_pos(p->A) || !finite_pos(p->cfl)) return WENOZN_EINVAL;
    if (!zn_constants_ok(p->eps, p->A)) return WENOZN_EINVAL;
    if (p->system == WENOZN_ADVECTION_1D) {
        if (!std::isfinite(p->adv_speed) || p->adv_speed == 0.0) return WENOZN_EINVAL;
    } else if (!std::isfinite(p->gamma) || p->gamma <= 1.0) {
        return WENOZN_EINVAL;
    }
    return WENOZN_OK;
}

inline wenozn_status cuda_status(cudaError_t e) { return e == cudaSuccess ? WENOZN_OK : WENOZN_ECUDA; }

inline FluxArgs flux_args(const wenozn_problem& p, const double* U, const unsigned long long* alpha_bits,
                          const unsigned long long* alpha_f_bits) {
    FluxArgs fa;
    fa.U = U;
    fa.alpha_bits = alpha_bits;
    fa.alpha_f_bits = alpha_f_bits;
    fa.weights = p.weights;
    fa.split = p.split;
    fa.nx = p.nx;
    fa.ny = p.ny;
    fa.eps4 = 4.0 * p.eps;
    fa.kappa = zn_kappa(p.A);
    fa.gamma = p.gamma;
    fa.adv_speed = p.adv_speed;
    fa.Fout = nullptr;
    fa.bc = p.bc_x;
    return fa;
}

// Launches the x (and y) flux kernels for stage input U with LF speeds in `alpha_bits`
// (and the per-field speeds in `alpha_f_bits`, [dir][3], for the per-field splitting).
inline cudaError_t launch_fluxes(const wenozn_problem& p, const double* U, const unsigned long long* alpha_bits,
                                 const unsigned long long* alpha_f_bits, double* fx, double* gy,
                                 cudaStream_t s) {
    FluxArgs fa = flux_args(p, U, alpha_bits, alpha_f_bits);
    fa.Fout = fx;
    if (p.system != WENOZN_EULER_2D) return launch_flux(p.system, 0, fa, s);
    FluxArgs fy = fa;
    fy.Fout = gy;
    fy.bc = p.bc_y;
    return launch_flux_xy(fa, fy, s);
}

inline UpdateArgs update_args(const wenozn_problem& p, Ctrl* ctrl, const double* fx, const double* gy) {
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
    u.clear_slot = -1;
    u.alpha_next = nullptr;
    u.field_speeds = p.split == WENOZN_SPLIT_LF_FIELD && p.system != WENOZN_ADVECTION_1D ? 1 : 0;
    u.cfl = p.cfl;
    u.dx = p.dx;
    u.dy = p.dy;
    u.gamma = p.gamma;
    u.adv_speed = p.adv_speed;
    return u;
}

inline char* ws_base(void* ws) { return static_cast<char*>(ws); }

// Clears every LF-speed slot (global and per-field) of the control block.
inline cudaError_t clear_speeds(Ctrl* ctrl, cudaStream_t s) {
    static_assert(offsetof(Ctrl, alpha_f) == sizeof(Ctrl::alpha), "speed slots must be adjacent");
    return cudaMemsetAsync(ctrl->alpha, 0, sizeof(Ctrl::alpha) + sizeof(Ctrl::alpha_f), s);
}

// The per-field speed slot to fill for this problem (null unless it splits per field).
inline unsigned long long* field_slot(const wenozn_problem& p, Ctrl* ctrl, int slot) {
    return p.split == WENOZN_SPLIT_LF_FIELD && p.system != WENOZN_ADVECTION_1D ? &ctrl->alpha_f[slot][0][0]
                                                                                : nullptr;
}

}  // namespace wz
