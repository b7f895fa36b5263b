// C ABI of libwenozn.so: argument checks, workspace layout and the launch sequences of
// the RHS evaluation and the SSP-RK3 step.  Declarations and contracts: include/wenozn.h.
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "host_common.h"

using namespace wz;


namespace wz {

namespace {
std::mutex g_status_mu;
std::unordered_map<void*, int32_t*> g_status_of_stream;   // stream -> device status word
}  // namespace

void note_status(void* stream, int32_t* status_dev) {
    std::lock_guard<std::mutex> lock(g_status_mu);
    g_status_of_stream[stream] = status_dev;
}

}  // namespace wz

namespace {

// The three SSP-RK3 stages: U1 = U + dt L(U), U2 = 3/4 U + 1/4 (U1 + dt L(U1)),
// U_out = 1/3 U + 2/3 (U2 + dt L(U2)); U_out may alias U.  The LF speeds of U, U1, U2 land in
// the control block's slots 0, 1, 2 and the step taken in its dt word.
cudaError_t rk3_stages(const wenozn_problem& p, const Layout& lay, void* ws, const double* U, double* U_out,
                       double* u1, double* u2, double dt, double t_remaining, cudaStream_t s) {
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws_base(ws) + lay.ctrl);
    double* fx = reinterpret_cast<double*>(ws_base(ws) + lay.fx);
    double* gy = reinterpret_cast<double*>(ws_base(ws) + lay.gy);
    const bool euler = p.system != WENOZN_ADVECTION_1D;
    cudaError_t e = clear_speeds(ctrl, s);
    if (e == cudaSuccess)
        e = launch_max_wavespeed(p.system, U, int64_t(p.nx) * p.ny, p.gamma, p.adv_speed, ctrl->alpha[0],
                                 &ctrl->status, s, field_slot(p, ctrl, 0));
    const double* stage_in[3] = {U, u1, u2};
    double* stage_out[3] = {u1, u2, U_out};
    for (int stage = 0; stage < 3 && e == cudaSuccess; ++stage) {
        e = launch_fluxes(p, stage_in[stage], ctrl->alpha[stage], &ctrl->alpha_f[stage][0][0], fx, gy, s);
        if (e != cudaSuccess) break;
        UpdateArgs u = update_args(p, ctrl, fx, gy);
        u.mode = stage + 1;
        u.Us = stage_in[stage];
        u.Un = U;
        u.out = stage_out[stage];
        u.next_slot = (euler && stage < 2) ? stage + 1 : -1;
        u.dt_fixed = dt;
        u.t_remaining = t_remaining;
        e = launch_update(p.system, u, s);
    }
    return e;
}

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
    p->weights = WENOZN_WEIGHTS_ZN;
    p->split = WENOZN_SPLIT_LF;
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
    if (!finite_pos(eps) || !finite_pos(A) || !zn_constants_ok(eps, A)) return WENOZN_EINVAL;
    return cuda_status(launch_reconstruct(f_padded, n, fhat, side, eps, A,
                                          static_cast<cudaStream_t>(stream)));
}

wenozn_status wenozn_reconstruct_weights(const double* f_padded, int64_t n, double* fhat, int32_t side,
                                         int32_t weights, double eps, double A, void* stream) {
    if (!f_padded || !fhat || n < 1 || n > (int64_t(1) << 31) - 8) return WENOZN_EINVAL;
    if (side != 1 && side != -1) return WENOZN_EINVAL;
    if (weights < 0 || weights > 3) return WENOZN_EINVAL;
    if (!finite_pos(eps) || !finite_pos(A) || !zn_constants_ok(eps, A)) return WENOZN_EINVAL;
    return cuda_status(launch_reconstruct(f_padded, n, fhat, side, eps, A, static_cast<cudaStream_t>(stream),
                                          weights));
}

wenozn_status wenozn_max_wavespeed(const wenozn_problem* p, const double* U, double* alpha_out,
                                   int32_t* status_dev, void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U || !alpha_out) return WENOZN_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool per_field = p->split == WENOZN_SPLIT_LF_FIELD && p->system != WENOZN_ADVECTION_1D;
    cudaError_t e = cudaMemsetAsync(alpha_out, 0, (per_field ? 8 : 2) * sizeof(double), s);
    if (e != cudaSuccess) return WENOZN_ECUDA;
    unsigned long long* a = reinterpret_cast<unsigned long long*>(alpha_out);
    return cuda_status(launch_max_wavespeed(p->system, U, int64_t(p->nx) * p->ny, p->gamma,
                                            p->adv_speed, a, status_dev, s, per_field ? a + 2 : nullptr));
}

wenozn_status wenozn_flux(const wenozn_problem* p, const double* U, const double* alpha,
                          int32_t dir, double* Fout, void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U || !Fout || U == Fout || (p->system != WENOZN_ADVECTION_1D && !alpha)) return WENOZN_EINVAL;
    if (dir != 0 && !((dir == 1 || dir == 2) && p->system == WENOZN_EULER_2D)) return WENOZN_EINVAL;
    FluxArgs fa;
    fa.U = U;
    fa.alpha_bits = reinterpret_cast<const unsigned long long*>(alpha);
    fa.alpha_f_bits = alpha ? fa.alpha_bits + 2 : nullptr;
    fa.weights = p->weights;
    fa.split = p->split;
    fa.nx = p->nx;
    fa.ny = p->ny;
    fa.eps4 = 4.0 * p->eps;
    fa.kappa = zn_kappa(p->A);
    fa.gamma = p->gamma;
    fa.adv_speed = p->adv_speed;
    fa.Fout = Fout;
    fa.bc = dir == 0 ? p->bc_x : p->bc_y;
    if (dir == 2) {
        // both sweeps in one launch, as wenozn_rhs and the RK3 steps run them
        FluxArgs fy = fa;
        fa.bc = p->bc_x;
        fy.Fout = Fout + int64_t(4) * p->ny * (int64_t(p->nx) + 1);
        return cuda_status(launch_flux_xy(fa, fy, static_cast<cudaStream_t>(stream)));
    }
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
    cudaError_t e = clear_speeds(ctrl, s);
    if (e == cudaSuccess)
        e = launch_max_wavespeed(p->system, U, int64_t(p->nx) * p->ny, p->gamma, p->adv_speed,
                                 ctrl->alpha[0], &ctrl->status, s, field_slot(*p, ctrl, 0));
    if (e == cudaSuccess) e = launch_fluxes(*p, U, ctrl->alpha[0], &ctrl->alpha_f[0][0][0], fx, gy, s);
    if (e == cudaSuccess) {
        UpdateArgs u = update_args(*p, ctrl, fx, gy);
        u.mode = 0;
        u.out = L;
        e = launch_update(p->system, u, s);
    }
    note_status(stream, &ctrl->status);
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
    note_status(stream, &ctrl->status);
    if (rk3_stages(*p, lay, ws, U, U, u1, u2, dt, t_remaining, s) != cudaSuccess) return WENOZN_ECUDA;
    if (dt_out) {
        cudaError_t e = cudaMemcpyAsync(dt_out, &ctrl->dt, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return WENOZN_ECUDA;
    }
    return WENOZN_OK;
}

wenozn_status wenozn_rk3_step_host(const wenozn_problem* p, const double* U_host_in, double* U_host_out,
                                   double* U_dev, double dt, double t_remaining, double* dt_out, void* ws,
                                   size_t ws_bytes, void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U_host_in || !U_host_out || !U_dev || !ws || std::isnan(dt) || std::isnan(t_remaining) || std::isinf(dt))
        return WENOZN_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return WENOZN_EINVAL;
    const Layout lay = layout_of(*p);
    if (ws_bytes < lay.total) return WENOZN_ENOMEM_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = size_t(nvar_of(p->system)) * size_t(p->nx) * size_t(p->ny) * sizeof(double);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws_base(ws) + lay.ctrl);
    double* u1 = reinterpret_cast<double*>(ws_base(ws) + lay.u1);
    double* u2 = reinterpret_cast<double*>(ws_base(ws) + lay.u2);
    note_status(stream, &ctrl->status);
    cudaError_t e = cudaMemcpyAsync(U_dev, U_host_in, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = rk3_stages(*p, lay, ws, U_dev, U_dev, u1, u2, dt, t_remaining, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(U_host_out, U_dev, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && dt_out) {
        e = cudaMemcpyAsync(dt_out, &ctrl->dt, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return cuda_status(e);
}

wenozn_status wenozn_rk3_stream_host(const wenozn_problem* p, int64_t count, const double* const* U_host_in,
                                     double* const* U_host_out, double* U_dev0, double* U_dev1, double dt, void* ws,
                                     size_t ws_bytes, void* stream, void* upload_stream, void* download_stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (count < 1 || !U_host_in || !U_host_out || !U_dev0 || !U_dev1 || U_dev0 == U_dev1 || !ws ||
        std::isnan(dt) || std::isinf(dt))
        return WENOZN_EINVAL;
    for (int64_t k = 0; k < count; ++k)
        if (!U_host_in[k] || !U_host_out[k]) return WENOZN_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return WENOZN_EINVAL;
    const Layout lay = layout_of(*p);
    if (ws_bytes < lay.total) return WENOZN_ENOMEM_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStream_t up = upload_stream ? static_cast<cudaStream_t>(upload_stream) : s;
    cudaStream_t down = download_stream ? static_cast<cudaStream_t>(download_stream) : s;
    const size_t bytes = size_t(nvar_of(p->system)) * size_t(p->nx) * size_t(p->ny) * sizeof(double);
    double* dev[2] = {U_dev0, U_dev1};
    double* u1 = reinterpret_cast<double*>(ws_base(ws) + lay.u1);
    double* u2 = reinterpret_cast<double*>(ws_base(ws) + lay.u2);
    note_status(stream, &reinterpret_cast<Ctrl*>(ws_base(ws) + lay.ctrl)->status);
    // ordering events of this call only: start, uploaded[2], stepped[2], downloaded[2]
    cudaEvent_t ev[7] = {};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 7 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    cudaEvent_t start = ev[0], *uploaded = ev + 1, *stepped = ev + 3, *downloaded = ev + 5;
    // the copy streams start after the work already on `stream`
    if (e == cudaSuccess) e = cudaEventRecord(start, s);
    if (e == cudaSuccess && up != s) e = cudaStreamWaitEvent(up, start, 0);
    if (e == cudaSuccess && down != s) e = cudaStreamWaitEvent(down, start, 0);
    for (int64_t k = 0; k < count && e == cudaSuccess; ++k) {
        const int b = int(k & 1);
        if (k >= 2) e = cudaStreamWaitEvent(up, downloaded[b], 0);            // the buffer is free again
        if (e == cudaSuccess) e = cudaMemcpyAsync(dev[b], U_host_in[k], bytes, cudaMemcpyHostToDevice, up);
        if (e == cudaSuccess) e = cudaEventRecord(uploaded[b], up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, uploaded[b], 0);
        if (e == cudaSuccess) e = rk3_stages(*p, lay, ws, dev[b], dev[b], u1, u2, dt, 0.0, s);
        if (e == cudaSuccess) e = cudaEventRecord(stepped[b], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(down, stepped[b], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(U_host_out[k], dev[b], bytes, cudaMemcpyDeviceToHost, down);
        if (e == cudaSuccess) e = cudaEventRecord(downloaded[b], down);
    }
    // `stream` ends after every copy of the call
    for (int b = 0; b < 2 && e == cudaSuccess; ++b)
        if (b < count) e = cudaStreamWaitEvent(s, downloaded[b], 0);
    for (int i = 0; i < 7; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);            // released once their pending work completes
    return cuda_status(e);
}

wenozn_status wenozn_cfl_dt(const wenozn_problem* p, const double* U, double* dt_out, void* ws, size_t ws_bytes,
                            void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U || !ws) return WENOZN_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return WENOZN_EINVAL;
    const Layout lay = layout_of(*p);
    if (ws_bytes < lay.total) return WENOZN_ENOMEM_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws_base(ws) + lay.ctrl);
    note_status(stream, &ctrl->status);
    cudaError_t e = clear_speeds(ctrl, s);
    if (e == cudaSuccess)
        e = launch_max_wavespeed(p->system, U, int64_t(p->nx) * p->ny, p->gamma, p->adv_speed, ctrl->alpha[0],
                                 &ctrl->status, s);
    if (e == cudaSuccess) {
        UpdateArgs u = update_args(*p, ctrl, nullptr, nullptr);
        e = launch_cfl_dt(p->system, u, s);
    }
    if (e == cudaSuccess && dt_out) {
        e = cudaMemcpyAsync(dt_out, &ctrl->dt, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return cuda_status(e);
}

wenozn_status wenozn_rk3_run(const wenozn_problem* p, double* U, int64_t nsteps, double dt, void* ws,
                             size_t ws_bytes, void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U || !ws || nsteps < 1 || std::isnan(dt) || std::isinf(dt)) return WENOZN_EINVAL;
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
    note_status(stream, &ctrl->status);
    // the speeds of U^n once; afterwards each step's last stage leaves those of U^{n+1} in
    // slot 0.  Stage s reads slot s, accumulates slot s+1 (mod 3) and clears slot s+2.
    cudaError_t e = clear_speeds(ctrl, s);
    if (e == cudaSuccess)
        e = launch_max_wavespeed(p->system, U, int64_t(p->nx) * p->ny, p->gamma, p->adv_speed, ctrl->alpha[0],
                                 &ctrl->status, s, field_slot(*p, ctrl, 0));
    const double* stage_in[3] = {U, u1, u2};
    double* stage_out[3] = {u1, u2, U};
    for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
        for (int stage = 0; stage < 3 && e == cudaSuccess; ++stage) {
            e = launch_fluxes(*p, stage_in[stage], ctrl->alpha[stage], &ctrl->alpha_f[stage][0][0], fx, gy, s);
            if (e != cudaSuccess) break;
            UpdateArgs u = update_args(*p, ctrl, fx, gy);
            u.mode = stage + 1;
            u.Us = stage_in[stage];
            u.Un = U;
            u.out = stage_out[stage];
            u.next_slot = euler ? (stage + 1) % 3 : -1;
            u.clear_slot = euler ? (stage + 2) % 3 : -1;
            u.dt_fixed = dt;
            e = launch_update(p->system, u, s);
        }
    }
    return cuda_status(e);
}

wenozn_status wenozn_rk3_step_keep(const wenozn_problem* p, const double* U, double* U_next, double dt,
                                   double* U1, double* U2, double* alphas, void* ws, size_t ws_bytes,
                                   void* stream) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!U || !U_next || !U1 || !U2 || !alphas || !ws || !(std::isfinite(dt) && dt > 0.0)) return WENOZN_EINVAL;
    if (U_next == U || U1 == U || U2 == U || U1 == U_next || U2 == U_next || U1 == U2) return WENOZN_EINVAL;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return WENOZN_EINVAL;
    const Layout lay = layout_of(*p);
    if (ws_bytes < lay.total) return WENOZN_ENOMEM_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws_base(ws) + lay.ctrl);
    note_status(stream, &ctrl->status);
    cudaError_t e = rk3_stages(*p, lay, ws, U, U_next, U1, U2, dt, 0.0, s);
    // the three stages' x speeds: alpha[s][0], s = 0, 1, 2 (a stride of two words)
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(alphas, sizeof(double), &ctrl->alpha[0][0], 2 * sizeof(unsigned long long),
                              sizeof(double), 3, cudaMemcpyDeviceToDevice, s);
    return cuda_status(e);
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

wenozn_status wenozn_last_error(void* stream, int32_t* device_status) {
    if (!device_status) return WENOZN_EINVAL;
    int32_t* dev = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_status_mu);
        auto it = g_status_of_stream.find(stream);
        if (it != g_status_of_stream.end()) dev = it->second;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t host = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && dev) e = cudaMemcpyAsync(&host, dev, sizeof host, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && dev) e = cudaMemsetAsync(dev, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return WENOZN_ECUDA;
    *device_status = host;
    return WENOZN_OK;
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
