// C ABI of the discrete adjoint (declarations and contracts in include/wenozn.h).
#include "host_common.h"

using namespace wz;

namespace {

VjpArgs vjp_args(const wenozn_problem& p, const Layout& L, void* ws) {
    VjpArgs v;
    std::memset(&v, 0, sizeof v);
    v.C = reinterpret_cast<double*>(ws_base(ws) + L.C);
    v.rec = v.C;
    v.rec_stride = vjp_rec_stride(p.nx);
    v.ctl = reinterpret_cast<unsigned*>(ws_base(ws) + L.vjp_ctl);
    v.prec[0] = v.prec[1] = v.prec[2] = -1;
    v.lam_slot = -1;
    v.x_slot[0] = v.x_slot[1] = v.x_slot[2] = -1;
    v.n = p.nx;
    v.bc = p.bc_x;
    v.rdx = 1.0 / p.dx;
    v.gamma = p.gamma;
    v.eps4 = 4.0 * p.eps;
    v.kappa = zn_kappa(p.A);
    v.adv_speed = p.adv_speed;
    return v;
}

wenozn_status check_vjp(const wenozn_problem* p, void* ws, size_t ws_bytes, Layout* L) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (p->system == WENOZN_EULER_2D) return WENOZN_EINVAL;     // the adjoint covers the 1D systems
    // ... of the default scheme (WENO-ZN weights, global LF, periodic or outflow boundaries)
    if (p->weights != WENOZN_WEIGHTS_ZN || p->split != WENOZN_SPLIT_LF || p->bc_x == WENOZN_BC_REFLECTIVE)
        return WENOZN_EINVAL;
    if (!ws || reinterpret_cast<uintptr_t>(ws) % kAlign) return WENOZN_EINVAL;
    *L = layout_of(*p);
    if (ws_bytes < L->total_vjp) return WENOZN_ENOMEM_WS;
    return WENOZN_OK;
}

// The state of a chain of Euler stage launches within one call: the launch count, the
// record each of lam, Ub2 and Ub1 still has pending (-1: none), and each record's d.
struct VjpChain {
    int t = 0;
    int lam_rec = -1, ub2_rec = -1, ub1_rec = -1;
    double d[kVjpRecs] = {};
};

// Sets up launch v of the chain: it writes record t mod kVjpRecs; `lam_rec` and the X_k
// records (-1: none; X_k == lam: read through lam's corrections) become pending slots.
void chain_launch(VjpChain& ch, VjpArgs& v, int lam_rec, const int x_rec[3], bool complete) {
    v.rec_out = ch.t % kVjpRecs;
    v.prec[0] = v.prec[1] = v.prec[2] = -1;
    int np = 0;
    auto slot_of = [&](int r) {
        if (r < 0) return -1;
        for (int q = 0; q < np; ++q)
            if (v.prec[q] == r) return q;
        v.prec[np] = r;
        return np++;
    };
    v.lam_slot = slot_of(lam_rec);
    const double* X[3] = {v.X1, v.X2, v.X3};
    for (int q = 0; q < 3; ++q) v.x_slot[q] = !X[q] ? -1 : (X[q] == v.lam ? -2 : slot_of(x_rec[q]));
    v.complete = complete ? 1 : 0;
    ch.d[v.rec_out] = v.d;
    for (int r = 0; r < kVjpRecs; ++r) v.rec_d[r] = ch.d[r];
    ++ch.t;
}

// Reverse of U3 = U0/3 + 2/3 (U2 + dt L(U2)), U2 = 3/4 U0 + 1/4 (U1 + dt L(U1)),
// U1 = U0 + dt L(U0), given the stage inputs and their LF speeds (bit patterns).  `last`:
// the call ends with this step, whose final launch completes in place.
wenozn_status reverse_stages(const wenozn_problem& p, const Layout& L, void* ws, const double* U0,
                             const double* U1, const double* U2, const unsigned long long* a0,
                             const unsigned long long* a1, const unsigned long long* a2, double dt,
                             double* lam, cudaStream_t s, VjpChain& ch, bool last) {
    double* ub2 = reinterpret_cast<double*>(ws_base(ws) + L.ub2);
    double* ub1 = reinterpret_cast<double*>(ws_base(ws) + L.ub1);
    VjpArgs v = vjp_args(p, L, ws);
    // the control words (argmax words, ticket counter) are zero before a chain starts
    cudaError_t e = ch.t == 0 ? cudaMemsetAsync(v.ctl, 0, (kVjpRecs + 1) * sizeof(unsigned), s) : cudaSuccess;
    if (e != cudaSuccess) return WENOZN_ECUDA;
    // Ub2 = 2/3 lam + 2/3 dt J(U2)^T lam
    v.U = U2; v.lam = lam; v.alpha_bits = a2; v.out = ub2;
    v.X1 = lam; v.c1 = 2.0 / 3.0; v.d = (2.0 / 3.0) * dt;
    const int none[3] = {-1, -1, -1};
    chain_launch(ch, v, ch.lam_rec, none, false);
    e = launch_vjp(p.system, v, s);
    ch.ub2_rec = v.rec_out;
    if (e == cudaSuccess) {                 // Ub1 = 1/4 Ub2 + 1/4 dt J(U1)^T Ub2
        v.U = U1; v.lam = ub2; v.alpha_bits = a1; v.out = ub1;
        v.X1 = ub2; v.c1 = 0.25; v.d = 0.25 * dt;
        chain_launch(ch, v, ch.ub2_rec, none, false);
        e = launch_vjp(p.system, v, s);
        ch.ub1_rec = v.rec_out;
    }
    if (e == cudaSuccess) {                 // lam <- lam/3 + 3/4 Ub2 + Ub1 + dt J(U0)^T Ub1
        v.U = U0; v.lam = ub1; v.alpha_bits = a0; v.out = lam;
        v.X1 = lam; v.c1 = 1.0 / 3.0; v.X2 = ub2; v.c2 = 0.75; v.X3 = ub1; v.c3 = 1.0; v.d = dt;
        const int xr[3] = {ch.lam_rec, ch.ub2_rec, -1};
        chain_launch(ch, v, ch.ub1_rec, xr, last);
        e = launch_vjp(p.system, v, s);
        ch.lam_rec = last ? -1 : v.rec_out;
    }
    return cuda_status(e);
}

}  // namespace

extern "C" {

wenozn_status wenozn_vjp_workspace_size(const wenozn_problem* p, size_t* bytes) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!bytes || p->system == WENOZN_EULER_2D) return WENOZN_EINVAL;
    if (p->weights != WENOZN_WEIGHTS_ZN || p->split != WENOZN_SPLIT_LF || p->bc_x == WENOZN_BC_REFLECTIVE)
        return WENOZN_EINVAL;
    *bytes = layout_of(*p).total_vjp;
    return WENOZN_OK;
}

wenozn_status wenozn_rhs_vjp(const wenozn_problem* p, const double* U, const double* lam, double* out,
                             void* ws, size_t ws_bytes, void* stream) {
    Layout L;
    wenozn_status st = check_vjp(p, ws, ws_bytes, &L);
    if (st != WENOZN_OK) return st;
    if (!U || !lam || !out || out == U || out == lam) return WENOZN_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws_base(ws) + L.ctrl);
    cudaError_t e = cudaMemsetAsync(ctrl->alpha, 0, sizeof(ctrl->alpha), s);
    if (e == cudaSuccess)
        e = launch_max_wavespeed(p->system, U, p->nx, p->gamma, p->adv_speed, ctrl->alpha[0], &ctrl->status, s);
    VjpArgs v = vjp_args(*p, L, ws);
    note_status(stream, &ctrl->status);
    if (e == cudaSuccess) e = cudaMemsetAsync(v.ctl, 0, (kVjpRecs + 1) * sizeof(unsigned), s);
    if (e == cudaSuccess) {
        v.U = U;
        v.lam = lam;
        v.alpha_bits = ctrl->alpha[0];
        v.out = out;
        v.d = 1.0;
        VjpChain ch;
        const int none[3] = {-1, -1, -1};
        chain_launch(ch, v, -1, none, true);
        e = launch_vjp(p->system, v, s);
    }
    return cuda_status(e);
}

wenozn_status wenozn_rk3_step_vjp(const wenozn_problem* p, const double* U, double dt, double* lam, void* ws,
                                  size_t ws_bytes, void* stream) {
    Layout L;
    wenozn_status st = check_vjp(p, ws, ws_bytes, &L);
    if (st != WENOZN_OK) return st;
    if (!U || !lam || U == lam || !(std::isfinite(dt) && dt > 0.0)) return WENOZN_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws_base(ws) + L.ctrl);
    double* u1 = reinterpret_cast<double*>(ws_base(ws) + L.u1);
    double* u2 = reinterpret_cast<double*>(ws_base(ws) + L.u2);
    double* fx = reinterpret_cast<double*>(ws_base(ws) + L.fx);
    double* ub2 = reinterpret_cast<double*>(ws_base(ws) + L.ub2);
    double* ub1 = reinterpret_cast<double*>(ws_base(ws) + L.ub1);
    const bool euler = p->system != WENOZN_ADVECTION_1D;

    // recompute the stage inputs U1, U2 of the forward step (same kernels, fixed dt)
    note_status(stream, &ctrl->status);
    cudaError_t e = cudaMemsetAsync(ctrl->alpha, 0, sizeof(ctrl->alpha), s);
    if (e == cudaSuccess)
        e = launch_max_wavespeed(p->system, U, p->nx, p->gamma, p->adv_speed, ctrl->alpha[0], &ctrl->status, s);
    const double* stage_in[2] = {U, u1};
    double* stage_out[2] = {u1, u2};
    for (int stage = 0; stage < 2 && e == cudaSuccess; ++stage) {
        e = launch_fluxes(*p, stage_in[stage], ctrl->alpha[stage], nullptr, fx, nullptr, s);
        if (e != cudaSuccess) break;
        UpdateArgs u = update_args(*p, ctrl, fx, nullptr);
        u.mode = stage + 1;
        u.Us = stage_in[stage];
        u.Un = U;
        u.out = stage_out[stage];
        u.next_slot = euler ? stage + 1 : -1;
        u.dt_fixed = dt;
        e = launch_update(p->system, u, s);
    }
    if (e != cudaSuccess) return WENOZN_ECUDA;
    const unsigned long long* a = &ctrl->alpha[0][0];
    VjpChain ch;
    return reverse_stages(*p, L, ws, U, u1, u2, a, a + 2, a + 4, dt, lam, s, ch, true);
}

wenozn_status wenozn_rk3_step_vjp_stages(const wenozn_problem* p, const double* U, const double* U1,
                                         const double* U2, const double* alphas, double dt, double* lam,
                                         void* ws, size_t ws_bytes, void* stream) {
    Layout L;
    wenozn_status st = check_vjp(p, ws, ws_bytes, &L);
    if (st != WENOZN_OK) return st;
    if (!U || !U1 || !U2 || !alphas || !lam || !(std::isfinite(dt) && dt > 0.0)) return WENOZN_EINVAL;
    if (lam == U || lam == U1 || lam == U2) return WENOZN_EINVAL;
    const unsigned long long* a = reinterpret_cast<const unsigned long long*>(alphas);
    VjpChain ch;
    return reverse_stages(*p, L, ws, U, U1, U2, a, a + 1, a + 2, dt, lam, static_cast<cudaStream_t>(stream), ch, true);
}

wenozn_status wenozn_workspace_stages(void* ws, const wenozn_problem* p, const double** U1, const double** U2,
                                      const double** alphas) {
    wenozn_status st = check_problem(p);
    if (st != WENOZN_OK) return st;
    if (!ws) return WENOZN_EINVAL;
    const Layout L = layout_of(*p);
    if (U1) *U1 = reinterpret_cast<const double*>(ws_base(ws) + L.u1);
    if (U2) *U2 = reinterpret_cast<const double*>(ws_base(ws) + L.u2);
    if (alphas) *alphas = reinterpret_cast<const double*>(&reinterpret_cast<Ctrl*>(ws_base(ws) + L.ctrl)->alpha[0][0]);
    return WENOZN_OK;
}

wenozn_status wenozn_rk3_run_keep(const wenozn_problem* p, double* X, double* S1, double* S2, double* alphas,
                                  int64_t nsteps, double dt, void* ws, size_t ws_bytes, void* stream) {
    Layout L;
    wenozn_status st = check_vjp(p, ws, ws_bytes, &L);
    if (st != WENOZN_OK) return st;
    if (!X || !S1 || !S2 || !alphas || nsteps < 1 || !(std::isfinite(dt) && dt > 0.0)) return WENOZN_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws_base(ws) + L.ctrl);
    double* fx = reinterpret_cast<double*>(ws_base(ws) + L.fx);
    const int64_t ns = int64_t(nvar_of(p->system)) * p->nx;          // one state
    unsigned long long* A = reinterpret_cast<unsigned long long*>(alphas);
    note_status(stream, &ctrl->status);
    // every speed accumulates into its own zeroed entry: A[k][s] for the stage-s input of step k
    cudaError_t e = cudaMemsetAsync(alphas, 0, size_t(3 * nsteps + 1) * sizeof(double), s);
    if (e == cudaSuccess)
        e = launch_max_wavespeed(p->system, X, p->nx, p->gamma, p->adv_speed, A, &ctrl->status, s);
    for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
        double* Xk = X + k * ns;
        const double* in[3] = {Xk, S1 + k * ns, S2 + k * ns};
        double* out[3] = {S1 + k * ns, S2 + k * ns, Xk + ns};
        for (int stage = 0; stage < 3 && e == cudaSuccess; ++stage) {
            e = launch_fluxes(*p, in[stage], A + 3 * k + stage, nullptr, fx, nullptr, s);
            if (e != cudaSuccess) break;
            UpdateArgs u = update_args(*p, ctrl, fx, nullptr);
            u.mode = stage + 1;
            u.Us = in[stage];
            u.Un = Xk;
            u.out = out[stage];
            u.alpha_next = p->system != WENOZN_ADVECTION_1D ? A + 3 * k + stage + 1 : nullptr;
            u.dt_fixed = dt;
            e = launch_update(p->system, u, s);
        }
    }
    return cuda_status(e);
}

wenozn_status wenozn_rk3_vjp_run(const wenozn_problem* p, const double* X, const double* S1, const double* S2,
                                 const double* alphas, int64_t nsteps, double dt, double* lam, void* ws,
                                 size_t ws_bytes, void* stream) {
    Layout L;
    wenozn_status st = check_vjp(p, ws, ws_bytes, &L);
    if (st != WENOZN_OK) return st;
    if (!X || !S1 || !S2 || !alphas || !lam || nsteps < 1 || !(std::isfinite(dt) && dt > 0.0)) return WENOZN_EINVAL;
    const int64_t ns = int64_t(nvar_of(p->system)) * p->nx;
    const unsigned long long* A = reinterpret_cast<const unsigned long long*>(alphas);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VjpChain ch;
    for (int64_t k = nsteps - 1; k >= 0; --k) {
        st = reverse_stages(*p, L, ws, X + k * ns, S1 + k * ns, S2 + k * ns, A + 3 * k, A + 3 * k + 1,
                            A + 3 * k + 2, dt, lam, s, ch, k == 0);
        if (st != WENOZN_OK) return st;
    }
    return WENOZN_OK;
}

}  // extern "C"
