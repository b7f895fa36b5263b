// Cell-wise kernels: flux difference + SSP-RK3 stage update (with the next stage's LF
// speeds folded in), the standalone LF-speed reduction, the single-line reconstruction and
// the ghost-cell fill.
#include "launch.h"
#include "speed_screen.cuh"

namespace wz {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double bits_to_double(unsigned long long b) {
    return __longlong_as_double((long long)b);
}

// CFL step of the current RK3 step from the LF speeds of U^n (slot 0), in the operation
// order of the oracle: 1D cfl dx / a_x (Sec. 4.3); 2D cfl dtx dty / (dtx + dty) with
// dtx = dx / a_x, dty = dy / a_y (Sec. 4.4); advection cfl dx / |a|.
__device__ __forceinline__ double step_dt(const UpdateArgs& a, int system) {
    double dt = a.dt_fixed;
    if (!(dt > 0.0)) {
        if (system == 0) {
            dt = __ddiv_rn(__dmul_rn(a.cfl, a.dx), fabs(a.adv_speed));
        } else {
            const double ax = bits_to_double(a.ctrl->alpha[0][0]);
            if (system == 1) {
                dt = __ddiv_rn(__dmul_rn(a.cfl, a.dx), ax);
            } else {
                const double ay = bits_to_double(a.ctrl->alpha[0][1]);
                const double tx = __ddiv_rn(a.dx, ax), ty = __ddiv_rn(a.dy, ay);
                dt = __ddiv_rn(__dmul_rn(__dmul_rn(a.cfl, tx), ty), __dadd_rn(tx, ty));
            }
        }
    }
    if (a.t_remaining > 0.0 && dt > a.t_remaining) dt = a.t_remaining;
    return dt;
}

// FIELDS: also the per-field speeds (per-field LF splitting), under the same screen
template <int NV, int T, bool FIELDS>
__global__ void __launch_bounds__(T, T >= 256 ? 4 : 1) update_kernel(UpdateArgs a) {
    pdl_wait();
    const int system = NV == 1 ? 0 : (NV == 3 ? 1 : 2);
    double dt = 0.0;
    if (a.mode == 1) {
        dt = step_dt(a, system);
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->dt = dt;
    } else if (a.mode > 1) {
        dt = a.ctrl->dt;
    }
    // the stage as base - kx dF - ky dG, with the RK weight of the update and dt/dx, dt/dy
    // folded into kx, ky: stage 1 U1 = U + dt L; 2: 3/4 U^n + 1/4 (U_s + dt L); 3: 1/3 U^n
    // + 2/3 (U_s + dt L), where L = -dF/dx - dG/dy (Eq. (2))
    const double wk = a.mode == 1 ? 1.0 : (a.mode == 2 ? 0.25 : 2.0 / 3.0);
    const double kx = wk * dt * a.rdx, ky = wk * dt * a.rdy;
    const int64_t nc = int64_t(a.nx) * a.ny;
    const int64_t sx = int64_t(a.ny) * (a.nx + 1);       // x-flux plane stride
    const int64_t sy = int64_t(a.ny + 1) * a.nx;         // y-flux plane stride
    double mx = 0.0, my = 0.0;
    double fmx[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // per-field speeds, x then y
    bool bad = false;
    // the next stage's LF speeds: exact evaluation only where the screen cannot rule a cell out
    const bool speeds = NV != 1 && a.mode != 0 && (a.next_slot >= 0 || a.alpha_next || a.mode == 3);
    // (64-thread blocks, used for small grids, hold two warps: one of them nearly always
    // holds the block's candidate, so they skip the screen)
    const bool screen = T >= 128 && speeds;
    const float gg1 = __double2float_rn(a.gamma * (a.gamma - 1.0));
    ScreenMax<T, FIELDS ? 8 : 2> smax;
    // the last state this thread evaluated exactly and its speeds: a bit-identical state
    // (constant regions) reuses them
    double cs[NV];
    double cvx = 0.0, cvy = 0.0;
    bool cached = false;
    // batches of T consecutive cells, the same count for every thread of the block; the row
    // j of the cell advances incrementally (one division per thread)
    const int64_t stride = int64_t(gridDim.x) * T;
    const int64_t dj = stride / a.nx, di = stride - dj * a.nx;
    int64_t j = (blockIdx.x * int64_t(T) + threadIdx.x) / a.nx;
    int64_t i = blockIdx.x * int64_t(T) + threadIdx.x - j * a.nx;
    for (int64_t base = blockIdx.x * int64_t(T); base < nc; base += stride) {
        const int64_t cell = base + threadIdx.x;
        const bool valid = cell < nc;
        const int64_t fx = cell + j;                      // j * (nx + 1) + i
        i += di;
        j += dj;
        if (i >= a.nx) {
            i -= a.nx;
            ++j;
        }
        double o[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            if (!valid) break;
            // Eq. (2): L = -(F^_{i+1/2} - F^_{i-1/2})/dx [- (G^_{j+1/2} - G^_{j-1/2})/dy]
            const double dF = a.Fx[k * sx + fx + 1] - a.Fx[k * sx + fx];
            const double dG = NV == 4 ? a.Gy[k * sy + cell + a.nx] - a.Gy[k * sy + cell] : 0.0;
            double r;
            if (a.mode == 0) {
                r = -(dF * a.rdx);
                if (NV == 4) r = fma(-dG, a.rdy, r);
                // a non-finite L (a stencil beyond the reconstruction's range): exponent test
                bad |= (__double2hiint(r) & 0x7ff00000) == 0x7ff00000;
            } else {
                const double us = a.Us[k * nc + cell];
                double base = us;
                if (a.mode == 2) base = fma(0.75, a.Un[k * nc + cell], 0.25 * us);
                else if (a.mode == 3) base = fma(1.0 / 3.0, a.Un[k * nc + cell], (2.0 / 3.0) * us);
                r = fma(-kx, dF, base);
                if (NV == 4) r = fma(-ky, dG, r);
            }
            a.out[k * nc + cell] = r;
            o[k] = r;
        }
        if (NV == 1) {
            if (a.mode != 0 && valid) bad |= !isfinite(o[0]);
        } else if (speeds) {
            bool exact = valid;
            if (screen) {
                SpeedEstimate est{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, true};
                if (valid) est = estimate_speeds<NV>(o, gg1);
                float e[FIELDS ? 8 : 2];
                e[0] = est.sx;
                e[1] = est.sy;
                if constexpr (FIELDS) estimate_field_speeds<NV>(est, e + 2);
                smax.add(e);
                bool cand = !est.ok || est.sx >= smax.m[0] * kScreenKeep ||
                            (NV == 4 && est.sy >= smax.m[1] * kScreenKeep);
                if constexpr (FIELDS) {
                    const float win = (1.0f - kScreenKeep) * fmaxf(smax.m[0], smax.m[1]);
#pragma unroll
                    for (int q = 2; q < (NV == 4 ? 8 : 5); ++q) cand = cand || e[q] >= smax.m[q] - win;
                }
                exact = valid && cand;
            }
            if (exact) {
                bool same = screen && cached;     // (a cached state's speeds are folded in already)
#pragma unroll
                for (int k = 0; k < NV; ++k) same = same && __double_as_longlong(o[k]) == __double_as_longlong(cs[k]);
                if (!same) {
                    double u, v, c;
                    const bool adm = wave_state<NV>(o, a.gamma, u, v, c);
                    cvx = __dadd_rn(fabs(u), c);
                    cvy = NV == 4 ? __dadd_rn(fabs(v), c) : 0.0;
                    bad |= !(adm && isfinite(cvx) && isfinite(cvy));
#pragma unroll
                    for (int k = 0; k < NV; ++k) cs[k] = o[k];
                    cached = true;
                    if (FIELDS) {
                        double f[3];
                        field_speeds(u, c, f);
                        for (int k = 0; k < 3; ++k) fmx[k] = fmax(fmx[k], f[k]);
                        if (NV == 4) {
                            field_speeds(v, c, f);
                            for (int k = 0; k < 3; ++k) fmx[3 + k] = fmax(fmx[3 + k], f[k]);
                        }
                    }
                }
                mx = fmax(mx, cvx);
                my = fmax(my, cvy);
            }
        }
    }
    if (bad) atomicOr(&a.ctrl->status, kStatusNonFinite);
    if (a.clear_slot >= 0 && blockIdx.x == 0 && threadIdx.x < 8) {
        unsigned long long* z = threadIdx.x < 2 ? &a.ctrl->alpha[a.clear_slot][threadIdx.x]
                                                : &a.ctrl->alpha_f[a.clear_slot][0][threadIdx.x - 2];
        *z = 0ull;
    }
    if (NV != 1 && a.alpha_next) {
        block_max2_atomic(mx, my, a.alpha_next, NV != 4);
    } else if (NV != 1 && a.next_slot >= 0) {
        block_max2_atomic(mx, my, a.ctrl->alpha[a.next_slot]);
        if (FIELDS) block_max_n_atomic<6>(fmx, &a.ctrl->alpha_f[a.next_slot][0][0]);
    }
}

// The CFL step of the LF speeds in slot 0 (one thread), the step the first RK stage takes.
__global__ void __launch_bounds__(32) cfl_dt_kernel(UpdateArgs a, int system) {
    if (threadIdx.x == 0) a.ctrl->dt = step_dt(a, system);
}

template <int NV, int T>
__global__ void __launch_bounds__(T) max_wavespeed_kernel(const double* U, int64_t nc, double gamma,
                                                          unsigned long long* dst, int32_t* status,
                                                          unsigned long long* dst_f) {
    double mx = 0.0, my = 0.0;
    double fmx[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    // the same screen as the update kernel's (exact evaluation only where it cannot rule a
    // cell out, bit-identical states reuse the last exact speeds)
    const bool screen = T >= 128 && dst_f == nullptr;
    const float gg1 = __double2float_rn(gamma * (gamma - 1.0));
    ScreenMax<T> smax;
    double cs[NV];
    bool cached = false;
    for (int64_t base = blockIdx.x * int64_t(T); base < nc; base += int64_t(gridDim.x) * T) {
        const int64_t cell = base + threadIdx.x;
        const bool valid = cell < nc;
        double s[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] = valid ? U[k * nc + cell] : 0.0;
        bool exact = valid;
        if (screen) {
            SpeedEstimate est{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, true};
            if (valid) est = estimate_speeds<NV>(s, gg1);
            const float e[2] = {est.sx, est.sy};
            smax.add(e);
            exact = valid && (!est.ok || est.sx >= smax.m[0] * kScreenKeep ||
                              (NV == 4 && est.sy >= smax.m[1] * kScreenKeep));
        }
        if (!exact) continue;
        bool same = screen && cached;
#pragma unroll
        for (int k = 0; k < NV; ++k) same = same && __double_as_longlong(s[k]) == __double_as_longlong(cs[k]);
        if (same) continue;
        double u, v, c;
        const bool adm = wave_state<NV>(s, gamma, u, v, c);
        const double vx = __dadd_rn(fabs(u), c), vy = NV == 4 ? __dadd_rn(fabs(v), c) : 0.0;
        bad |= !(adm && isfinite(vx) && isfinite(vy));
        mx = fmax(mx, vx);
        my = fmax(my, vy);
#pragma unroll
        for (int k = 0; k < NV; ++k) cs[k] = s[k];
        cached = true;
        if (dst_f) {
            double f[3];
            field_speeds(u, c, f);
            for (int k = 0; k < 3; ++k) fmx[k] = fmax(fmx[k], f[k]);
            if (NV == 4) {
                field_speeds(v, c, f);
                for (int k = 0; k < 3; ++k) fmx[3 + k] = fmax(fmx[3 + k], f[k]);
            }
        }
    }
    if (bad && status) atomicOr(status, kStatusNonFinite);
    block_max2_atomic(mx, my, dst);
    if (dst_f) block_max_n_atomic<6>(fmx, dst_f);
}

__global__ void __launch_bounds__(kThreads) abs_speed_kernel(double adv_speed, unsigned long long* dst) {
    if (threadIdx.x == 0) {
        dst[0] = (unsigned long long)__double_as_longlong(fabs(adv_speed));
        dst[1] = 0ull;
    }
}

// WENO-ZN weights, a tile of kThreads interfaces a block: the first differences
// D_i = f_i - f_{i+1} and the second-difference part of the indicators,
// S_i = (13/3)(D_i - D_{i+1})^2 + 4 eps, are shared by neighbouring interfaces (sub-stencil k of
// interface j covers f_{j+k} .. f_{j+k+2}, mirrored for the minus side), so each is formed once
// per point in shared memory; the one-sided parts of the indicators differ between the
// sub-stencils and stay per interface.  The minus side's mirrored stencil has the negated
// differences in reverse order.
__global__ void __launch_bounds__(kThreads) reconstruct_zn_kernel(const double* f, int64_t n, double* fhat,
                                                                   int side, double eps4, double kappa) {
    __shared__ double sf[kThreads + 5], sD[kThreads + 4], sS[kThreads + 3];
    const int64_t j0 = blockIdx.x * int64_t(kThreads);
    const int tid = threadIdx.x;
    for (int t = tid; t < kThreads + 5; t += kThreads) {
        const int64_t g = j0 + t;
        sf[t] = g < n + 6 ? f[g] : 0.0;
    }
    __syncthreads();
    for (int t = tid; t < kThreads + 4; t += kThreads) sD[t] = sf[t] - sf[t + 1];
    __syncthreads();
    const double k13_3 = 13.0 / 3.0;
    for (int t = tid; t < kThreads + 3; t += kThreads) {
        const double s2 = sD[t] - sD[t + 1];
        sS[t] = fma(k13_3 * s2, s2, eps4);
    }
    __syncthreads();
    const int64_t j = j0 + tid;
    if (j > n) return;
    const int i = tid;
    fhat[j] = side > 0 ? zn_flux_ds(sD[i], sD[i + 1], sD[i + 2], sD[i + 3], sS[i], sS[i + 1], sS[i + 2], sf[i + 2],
                                    eps4, kappa)
                       : zn_flux_ds<true>(sD[i + 4], sD[i + 3], sD[i + 2], sD[i + 1], sS[i + 3], sS[i + 2],
                                          sS[i + 1], sf[i + 3], eps4, kappa);   // the mirrored stencil
}

__global__ void __launch_bounds__(kThreads) reconstruct_kernel(const double* f, int64_t n, double* fhat,
                                                                int side, double eps4, double kappa,
                                                                int weights) {
    const int64_t j = blockIdx.x * int64_t(kThreads) + threadIdx.x;
    if (j > n) return;
    const double* s = f + j;
    fhat[j] = side > 0 ? zn_flux_w(s[0], s[1], s[2], s[3], s[4], eps4, kappa, weights)
                       : zn_flux_w(s[5], s[4], s[3], s[2], s[1], eps4, kappa, weights);
}

// x-ghosts of the interior rows (phase 0) or y-ghosts of every padded column (phase 1).
__global__ void __launch_bounds__(kThreads) ghost_kernel(double* U, int nv, int nx, int ny, int bc_x,
                                                          int bc_y, int two_d, int phase) {
    const int px = nx + 6, py = two_d ? ny + 6 : 1;
    const int64_t t = blockIdx.x * int64_t(kThreads) + threadIdx.x;
    if (phase == 0) {
        const int rows = two_d ? ny : 1;
        const int64_t total = int64_t(nv) * rows * 6;
        if (t >= total) return;
        const int g = int(t % 6);
        const int64_t r = (t / 6) % rows, k = t / (6 * int64_t(rows));
        const int64_t row = two_d ? r + 3 : 0;
        double* line = U + (k * py + row) * px;
        const int gi = g < 3 ? g - 3 : nx + (g - 3);          // -3..-1, n..n+2
        const double val = line[ghost_src(gi, nx, bc_x) + 3];
        // a wall's mirror image carries the opposite x momentum
        line[gi + 3] = (nv > 1 && k == 1 && ghost_mirrored(gi, nx, bc_x)) ? -val : val;
    } else {
        const int64_t total = int64_t(nv) * px * 6;
        if (t >= total) return;
        const int g = int(t % 6);
        const int64_t col = (t / 6) % px, k = t / (6 * int64_t(px));
        double* plane = U + k * py * px;
        const int gj = g < 3 ? g - 3 : ny + (g - 3);
        const double val = plane[int64_t(ghost_src(gj, ny, bc_y) + 3) * px + col];
        plane[int64_t(gj + 3) * px + col] = (k == 2 && ghost_mirrored(gj, ny, bc_y)) ? -val : val;
    }
}

unsigned grid_for(int64_t items, int cap, int threads = kThreads) {
    int64_t b = (items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return unsigned(b);
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 152;
    return sms > 0 ? sms : 152;
}

}  // namespace

// The per-cell kernels are FP64-pipe bound: with fewer than two 256-thread blocks per SM
// they run 64-thread blocks instead, so that the work spreads over all SMs.
bool few_cells(int64_t nc, int sms) { return nc < int64_t(sms) * 2 * kThreads; }

// Blocks of `kern` resident on one SM at once: the grid-stride kernels launch exactly that
// many per SM, so that every SM gets the same number of cells (no partial last wave).
template <typename... KArgs>
int resident_blocks(void (*kern)(KArgs...), int threads) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, 0) != cudaSuccess || n < 1) n = 1;
    return n;
}

template <int NV, bool FIELDS>
void update_nv(const UpdateArgs& a, int64_t nc, cudaStream_t s) {
    const int sms = sm_count();
    static const int occ = resident_blocks(update_kernel<NV, kThreads, FIELDS>, kThreads);
    if (few_cells(nc, sms))
        launch_pdl(update_kernel<NV, 64, FIELDS>, dim3(grid_for(nc, sms * 32, 64)), dim3(64), 0, s, a);
    else
        launch_pdl(update_kernel<NV, kThreads, FIELDS>, dim3(grid_for(nc, sms * occ)), dim3(kThreads), 0, s, a);
}

template <int NV>
void max_wavespeed_nv(const double* U, int64_t nc, double gamma, unsigned long long* dst, int32_t* status,
                      unsigned long long* dst_f, cudaStream_t s) {
    const int sms = sm_count();
    static const int occ = resident_blocks(max_wavespeed_kernel<NV, kThreads>, kThreads);
    if (few_cells(nc, sms))
        max_wavespeed_kernel<NV, 64><<<grid_for(nc, sms * 16, 64), 64, 0, s>>>(U, nc, gamma, dst, status, dst_f);
    else
        max_wavespeed_kernel<NV, kThreads><<<grid_for(nc, sms * occ), kThreads, 0, s>>>(U, nc, gamma, dst, status,
                                                                                          dst_f);
}

cudaError_t launch_update(int system, const UpdateArgs& a, cudaStream_t s) {
    const int64_t nc = int64_t(a.nx) * a.ny;
    if (system == 0) update_nv<1, false>(a, nc, s);
    else if (system == 1) a.field_speeds ? update_nv<3, true>(a, nc, s) : update_nv<3, false>(a, nc, s);
    else a.field_speeds ? update_nv<4, true>(a, nc, s) : update_nv<4, false>(a, nc, s);
    return cudaGetLastError();
}

cudaError_t launch_cfl_dt(int system, const UpdateArgs& a, cudaStream_t s) {
    cfl_dt_kernel<<<1, 32, 0, s>>>(a, system);
    return cudaGetLastError();
}

cudaError_t launch_max_wavespeed(int system, const double* U, int64_t ncells, double gamma,
                                 double adv_speed, unsigned long long* dst, int32_t* status,
                                 cudaStream_t s, unsigned long long* dst_f) {
    if (system == 0) {
        abs_speed_kernel<<<1, 32, 0, s>>>(adv_speed, dst);
        return cudaGetLastError();
    }
    if (system == 1) max_wavespeed_nv<3>(U, ncells, gamma, dst, status, dst_f, s);
    else max_wavespeed_nv<4>(U, ncells, gamma, dst, status, dst_f, s);
    return cudaGetLastError();
}

cudaError_t launch_reconstruct(const double* f_padded, int64_t n, double* fhat, int side,
                               double eps, double A, cudaStream_t s, int weights) {
    const unsigned grid = unsigned((n + 1 + kThreads - 1) / kThreads);
    if (weights == 0)
        reconstruct_zn_kernel<<<grid, kThreads, 0, s>>>(f_padded, n, fhat, side, 4.0 * eps, zn_kappa(A));
    else
        reconstruct_kernel<<<grid, kThreads, 0, s>>>(f_padded, n, fhat, side, 4.0 * eps, zn_kappa(A), weights);
    return cudaGetLastError();
}

cudaError_t launch_fill_ghosts(int nv, int nx, int ny, int bc_x, int bc_y, int two_d,
                               double* U_padded, cudaStream_t s) {
    const int64_t t0 = int64_t(nv) * (two_d ? ny : 1) * 6;
    ghost_kernel<<<unsigned((t0 + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        U_padded, nv, nx, ny, bc_x, bc_y, two_d, 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !two_d) return e;
    const int64_t t1 = int64_t(nv) * (nx + 6) * 6;
    ghost_kernel<<<unsigned((t1 + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        U_padded, nv, nx, ny, bc_x, bc_y, two_d, 1);
    return cudaGetLastError();
}

}  // namespace wz
