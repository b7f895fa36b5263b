// Internal host-side launchers shared by the translation units of libwenozn.so.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "wenozn_device.cuh"

namespace wz {

// Launches a kernel that begins with pdl_wait() with programmatic stream serialization
// allowed, so that it can be scheduled while the previous kernel in the stream finishes
// (a memset or copy before it is waited for as usual).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Numerical fluxes at every interface of one sweep direction.
//   dir 0 (x): Fout[nv][ny][nx+1], Fout[.][j][i] at x_{i-1/2} of row j.
//   dir 1 (y): Fout[nv][ny+1][nx], Fout[.][j][i] at y_{j-1/2} of column i.
struct FluxArgs {
    const double* U;                       // stage input, [nv][ny][nx]
    double* Fout;
    const unsigned long long* alpha_bits;  // LF speeds (x, y) of U as bit patterns; unused for advection
    const unsigned long long* alpha_f_bits;  // per-field speeds [dir][3] (split 1 only)
    int nx, ny, bc;                        // bc of the sweep direction (0 periodic, 1 outflow, 2 reflective)
    int weights, split;                    // weight function and flux splitting (wenozn.h enums)
    double eps4, kappa, gamma, adv_speed;  // eps4 = 4 eps, kappa = 2 / sqrt(A) (see zn_parts)
};
// Admissible constants of the weights: with 1e-60 <= eps <= 1 and 1e-6 <= A <= 1e6 the
// reconstruction's common denominator is a positive normal number and its range guard
// (zn_flux) covers every stencil whose differences stay below 2^440.
inline bool zn_constants_ok(double eps, double A) {
    return eps >= 1e-60 && eps <= 1.0 && A >= 1e-6 && A <= 1e6;
}
// The WENO-ZN weights carry A as kappa = 2 / sqrt(A) (A > 0, checked on entry).
inline double zn_kappa(double A) { return 2.0 / std::sqrt(A); }
cudaError_t launch_flux(int system, int dir, const FluxArgs& a, cudaStream_t s);
// both sweeps of a 2D stage (x fluxes into ax.Fout, y fluxes into ay.Fout) in one launch
cudaError_t launch_flux_xy(const FluxArgs& ax, const FluxArgs& ay, cudaStream_t s);

// Flux difference, SSP-RK3 stage combination and the next stage's LF speeds.
struct UpdateArgs {
    const double* Us;    // stage input
    const double* Un;    // state at the start of the step (stages 1 and 2)
    double* out;         // stage output (may alias Un for the last stage), or L (mode 0)
    const double* Fx;
    const double* Gy;    // null in 1D
    int nx, ny;
    double rdx, rdy;     // 1/dx, 1/dy
    int mode;            // 0: out = L; 1, 2, 3: RK3 stages
    Ctrl* ctrl;
    int next_slot;       // alpha slot to accumulate the output's LF speeds into, or -1
    int field_speeds;    // also accumulate the per-field speeds (per-field LF splitting)
    int clear_slot;      // alpha slot to zero (a later stage accumulates into it), or -1
    unsigned long long* alpha_next;   // if set: accumulate the output's LF speed here instead of a slot
    double dt_fixed, t_remaining, cfl, dx, dy, gamma, adv_speed;
};
cudaError_t launch_update(int system, const UpdateArgs& a, cudaStream_t s);
// ctrl->dt = the CFL step of the LF speeds in ctrl->alpha[0] (a.dt_fixed <= 0, no clipping
// unless a.t_remaining > 0), in the update kernel's operation order.
cudaError_t launch_cfl_dt(int system, const UpdateArgs& a, cudaStream_t s);

// Global LF speeds of U folded into dst[0..1] (bit-pattern max; dst must start at 0) and,
// when dst_f is not null, the per-field speeds into dst_f[dir][3] (|u-c|, |u|, |u+c|).
cudaError_t launch_max_wavespeed(int system, const double* U, int64_t ncells, double gamma,
                                 double adv_speed, unsigned long long* dst, int32_t* status,
                                 cudaStream_t s, unsigned long long* dst_f = nullptr);

cudaError_t launch_reconstruct(const double* f_padded, int64_t n, double* fhat, int side,
                               double eps, double A, cudaStream_t s, int weights = 0);

// Batched 1D Euler (see batch_kernels.cu).
struct BatchArgs {
    const double* Us;          // stage input, [3][total]
    const double* Un;          // state at the start of the step
    double* out;               // stage output (aliases Un in the last stage)
    int64_t total;             // plane stride: total cells of the batch
    int B;                     // instances
    const int64_t* off;        // [B+1] first cell of each instance
    const int32_t* tile_off;   // [B+1] prefix count of tiles (tiles of TI-1 cells)
    const double* dx;          // [B]
    unsigned long long* alpha; // [3][B] LF speeds per stage slot, bit patterns
    double* dt;                // [B] step of the current RK3 step
    double* t;                 // [B] time reached
    int32_t* status;
    int stage;                 // 0, 1, 2
    int bc;                    // ghost map of every instance
    double gamma, eps4, kappa, cfl;
    double t_final;            // > 0: no instance steps past it
};
struct BatchShape { int tile, threads; };
constexpr int kNumBatchShapes = 5;
extern const BatchShape kBatchShapes[kNumBatchShapes];
cudaError_t batch_configure();
cudaError_t launch_batch_init(const BatchArgs& a, cudaStream_t s);
cudaError_t launch_batch_stage(int shape, const BatchArgs& a, int sms, cudaStream_t s);

// Adjoint of the 1D right-hand side (see adjoint_kernels.cu).
// The Euler stage kernel's correction records: a ring of kVjpRecs (a launch's record is
// read by the launches up to three stages later, and cleared by the one after those), and
// at most kVjpPend records pending on one launch's inputs.
constexpr int kVjpRecs = 5;
constexpr int kVjpPend = 3;

struct VjpArgs {
    const double* U;                       // stage input, [nv][n]
    const double* lam;                     // cotangent of L(U), [nv][n]
    double* C;                             // advection: per-interface contributions, vjp_contrib_doubles(1, n)
    double* rec;                           // Euler: kVjpRecs correction records of rec_stride doubles
    int64_t rec_stride;
    unsigned* ctl;                         // ctl[r]: ~(argmax of the LF speed) of record r, ctl[kVjpRecs]:
                                           // ticket counter of a completing launch; zero when unused
    const unsigned long long* alpha_bits;  // LF speed of U (bit pattern)
    double* out;                           // c1 X1 + c2 X2 + c3 X3 + d J^T lam
    const double* X1;
    const double* X2;
    const double* X3;
    double c1, c2, c3, d;
    int n, bc;
    double rdx, gamma, eps4, kappa, adv_speed;
    int rec_out;                           // the record this launch writes
    int prec[kVjpPend];                    // records with corrections pending on the inputs (-1: none)
    int lam_slot;                          // index into prec of lam's record (-1: none)
    int x_slot[3];                         // ... of X1..X3 (-1: none; -2: X_t is lam itself)
    int complete;                          // apply this launch's own record in place (a call's last launch)
    double rec_d[kVjpRecs];                // d of the launch that wrote each record
};
int64_t vjp_rec_stride(int n);
size_t vjp_contrib_doubles(int nv, int n);
cudaError_t launch_vjp(int system, const VjpArgs& a, cudaStream_t s);

// Remembers the device status word the most recent stepping call on `stream` wrote to
// (read back by wenozn_last_error).
void note_status(void* stream, int32_t* status_dev);

cudaError_t launch_fill_ghosts(int nv, int nx, int ny, int bc_x, int bc_y, int two_d,
                               double* U_padded, cudaStream_t s);

}  // namespace wz
