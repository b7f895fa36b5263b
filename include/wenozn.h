/*
 * wenozn.h - C ABI of the GB300 (sm_103a) WENO-ZN finite-difference solver.
 *
 * The library implements the fifth-order WENO-ZN scheme of Shen, Zhang, Li & Peng,
 * "A novel method for constructing high accurate and robust WENO-Z type scheme"
 * (arXiv 2004.07954), inside an SSP-RK3 solver for linear advection and the 1D / 2D Euler
 * equations, all in FP64.  Section and equation labels below are the paper's.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers documented as "device" must point to CUDA global memory of the current
 *    device; "host" pointers to ordinary or pinned host memory.  The caller owns every
 *    buffer; the library allocates nothing on these paths and keeps no pointer after a
 *    call returns.  Scratch space comes from the caller's workspace (wenozn_workspace_size).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Every
 *    call only enqueues work on it and returns; the only calls that synchronise are the
 *    ones that say so (a non-NULL host `dt_out`, wenozn_workspace_status).
 *  - State arrays are FP64, planar and C-contiguous: U[nvar][ny][nx], x fastest, holding
 *    the conserved variables (rho, rho u, E) in 1D, (rho, rho u, rho v, E) in 2D, or the
 *    scalar u for advection.  1D problems use ny = 1.
 *  - Host-side argument checks run first and return WENOZN_EINVAL without enqueuing
 *    anything.  Launch failures return WENOZN_ECUDA.  Conditions detected on the device
 *    (non-finite values, rho <= 0 or p <= 0) set bits in the workspace status word, read
 *    with wenozn_workspace_status; the kernels never trap.
 *  - Range of the reconstruction.  The weights are evaluated division-free (their common
 *    denominator is a fifth-degree product of the smoothness indicators).  When that
 *    product leaves the double range (stencil differences above about 1e26, or data far
 *    below the scale of eps), the weights are evaluated again on the stencil scaled by an
 *    exact power of two, which is exact algebra.  With the admissible constants
 *    (1e-60 <= eps <= 1, 1e-6 <= A <= 1e6; other values return WENOZN_EINVAL) every
 *    reconstruction is therefore finite and accurate to rounding for stencils whose first
 *    differences stay below 2^440 (about 2.8e132) in magnitude; for Euler these are the
 *    differences of the split characteristic fluxes.  Beyond that bound (where the plain
 *    evaluation of Eq. (new) itself overflows: tau8 / eps exceeds the double range) results
 *    may be non-finite, which the stepping calls report as WENOZN_ENONFINITE.
 */
#ifndef WENOZN_H
#define WENOZN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WENOZN_OK = 0,
    WENOZN_EINVAL = 1,       /* bad argument (null pointer, size, enum, non-positive dx ...) */
    WENOZN_ECUDA = 2,        /* a CUDA launch or copy failed                                 */
    WENOZN_ENOMEM_WS = 3,    /* workspace smaller than wenozn_workspace_size reports         */
    WENOZN_ENONFINITE = 4,   /* device status bit: NaN/Inf, rho <= 0 or p <= 0 encountered   */
    WENOZN_ETIMEOUT = 5      /* device status bit: a bounded device-side wait gave up        */
} wenozn_status;

/* Boundary conditions: periodic (Sec. 4.2); outflow, the zero-order extrapolation of the
 * transmissive condition (Sec. 4.4); reflective wall (the blast-wave and Rayleigh-Taylor
 * set-ups of Sec. 4.3.2 / 4.4): ghost cell -1-g (g < 0) or 2n-1-g (g >= n) with the momentum
 * normal to the wall negated (for advection the mirror image alone). */
typedef enum { WENOZN_BC_PERIODIC = 0, WENOZN_BC_OUTFLOW = 1, WENOZN_BC_REFLECTIVE = 2 } wenozn_bc;

/* Weight function of the fifth-order reconstruction: WENO-ZN (Eq. (new), the method),
 * WENO-Z with q = 1 (Eq. (15)), the linear optimal weights c_k, or Jiang-Shu
 * (alpha_k = c_k / (IS_k + eps)^2, Sec. 2.1; the paper's JS runs use eps = 1e-6). */
typedef enum {
    WENOZN_WEIGHTS_ZN = 0, WENOZN_WEIGHTS_Z = 1, WENOZN_WEIGHTS_LINEAR = 2, WENOZN_WEIGHTS_JS = 3
} wenozn_weights;

/* Flux splitting (Euler; advection always splits with |a|): global Lax-Friedrichs, one
 * speed per direction (Sec. 4.3, the default); global LF with one speed per characteristic
 * field, max |u - c|, max |u|, max |u + c|; local LF with the largest |u| + c of each
 * interface's six stencil cells; Steger-Warming flux-vector splitting (Sec. 4.4). */
typedef enum {
    WENOZN_SPLIT_LF = 0, WENOZN_SPLIT_LF_FIELD = 1, WENOZN_SPLIT_LLF = 2, WENOZN_SPLIT_SW = 3
} wenozn_split;

typedef enum {
    WENOZN_ADVECTION_1D = 0, /* u_t + a u_x = 0 (Sec. 4.2), nvar = 1 */
    WENOZN_EULER_1D = 1,     /* Sec. 4.3, nvar = 3                  */
    WENOZN_EULER_2D = 2      /* Sec. 4.4, nvar = 4                  */
} wenozn_system;

/* Problem description.  The numerical constants default to the paper's choices:
 * gamma = 1.4 (Sec. 4.3), eps = 1e-40 in Eq. (new) (the value that reproduces the Sec. 4.1
 * table), A = 10 in Eq. (function), cfl = 0.5 (Sec. 4), WENO-ZN weights, global LF
 * splitting.  `flags` must be 0. */
typedef struct {
    int32_t system;          /* wenozn_system                                  */
    int32_t nx, ny;          /* interior cells, 1 .. 2^30 each, nx*ny <= 2^34; ny = 1 in 1D */
    int32_t bc_x, bc_y;      /* wenozn_bc per direction (bc_y ignored in 1D)   */
    int32_t weights;         /* wenozn_weights                                 */
    int32_t split;           /* wenozn_split                                   */
    int32_t flags;           /* reserved, 0                                    */
    double dx, dy;           /* uniform spacing (> 0; dy ignored in 1D)        */
    double gamma;            /* ratio of specific heats (Euler)                */
    double eps;              /* epsilon of Eq. (function) / Eq. (new), 1e-60 .. 1 */
    double A;                /* constant A of Eq. (function), 1e-6 .. 1e6      */
    double cfl;              /* CFL number sigma of the time-step formulas     */
    double adv_speed;        /* advection speed a (advection only)             */
} wenozn_problem;

/* Fills `p` with the paper's defaults for `system` on an nx x ny grid of spacing dx, dy,
 * outflow boundaries.  Returns WENOZN_EINVAL for a null pointer or unknown system. */
wenozn_status wenozn_problem_init(wenozn_problem* p, int32_t system, int32_t nx, int32_t ny,
                                  double dx, double dy);

/* Bytes of caller-provided device workspace that wenozn_rhs / wenozn_rk3_step need for
 * this problem: a 256-byte control block (LF speeds, time step, status word), two
 * state-sized RK stage buffers and the interface fluxes of each sweep direction
 * ([nvar][ny][nx+1], and [nvar][ny+1][nx] in 2D), each region 256-byte aligned.  The
 * workspace must be 256-byte aligned and zero-filled once before its first use
 * (cudaMemset); the library keeps it consistent afterwards.  Returns WENOZN_EINVAL for an
 * invalid problem or a null `bytes`. */
wenozn_status wenozn_workspace_size(const wenozn_problem* p, size_t* bytes);

/* Ghost-cell fill (three cells per side).  Periodic boundaries wrap (Sec. 4.2: "periodic
 * boundary"); outflow boundaries copy the edge cell (zero-order extrapolation, the
 * transmissive condition named in Sec. 4.4).
 *   U_padded : device, FP64, [nvar][ny+6][nx+6] in 2D or [nvar][nx+6] in 1D, interior at
 *              offset 3 in each padded direction; ghosts are overwritten in place.  In 2D
 *              the x-ghosts of the interior rows are filled first, then the y-ghosts of
 *              every padded column (so corners hold the doubly extrapolated values). */
wenozn_status wenozn_fill_ghosts(const wenozn_problem* p, double* U_padded, void* stream);

/* Fifth-order WENO-ZN reconstruction of one padded line (Sec. 3, Eqs. (3), (4), (isjiang),
 * (tau), (tau8), (function), (new)).
 *   f_padded : device, n + 6 values, f_padded[j + 3] = f_j, ghosts already filled.
 *   n        : interior points, 1 <= n <= 2^31 - 8.
 *   fhat     : device, n + 1 values; fhat[j] is the flux at x_{j-1/2}, j = 0..n.
 *   side     : +1 for f^+_{j-1/2} (stencil f_{j-3..j+1}); -1 for f^-_{j-1/2}, the same
 *              formula applied to the mirrored stencil (f_{j+2}, f_{j+1}, f_j, f_{j-1},
 *              f_{j-2}) (Sec. 2: "symmetric rule about x_{i+1/2}").
 *   eps, A   : Eq. (function) / (new) constants, 1e-60 <= eps <= 1 and 1e-6 <= A <= 1e6
 *              (WENOZN_EINVAL otherwise).  Finite and accurate for stencils whose first
 *              differences stay below 2^440 (see "Range of the reconstruction" above). */
wenozn_status wenozn_reconstruct(const double* f_padded, int64_t n, double* fhat, int32_t side,
                                 double eps, double A, void* stream);

/* The same reconstruction with the weight function `weights` (wenozn_weights); A is used by
 * WENO-ZN only.  EINVAL for an unknown weight function. */
wenozn_status wenozn_reconstruct_weights(const double* f_padded, int64_t n, double* fhat, int32_t side,
                                         int32_t weights, double eps, double A, void* stream);

/* Global Lax-Friedrichs speeds (Sec. 4.3 / 4.4): alpha_out[0] = max_ij(|u| + c),
 * alpha_out[1] = max_ij(|v| + c) (2D; 0 otherwise); |a| for advection.  With the per-field
 * splitting also alpha_out[2..4] = max |u - c|, max |u|, max |u + c| and alpha_out[5..7] the
 * same with v (2D; 0 otherwise).  The maxima are those of the per-cell speeds evaluated with
 * IEEE operations in the order u = m/rho, p = (gamma-1)(E - rho u^2/2), c = sqrt(gamma p/rho)
 * (bit-identical whatever the grid's decomposition; a single-precision estimate with a
 * proven error bound only decides which cells need that evaluation).
 *   U         : device state [nvar][ny][nx].
 *   alpha_out : device, 2 doubles (8 with the per-field splitting), overwritten.
 *   status_dev: device int32 status word or NULL; a NaN/Inf, rho <= 0 or p <= 0 ORs
 *               WENOZN_ENONFINITE into it. */
wenozn_status wenozn_max_wavespeed(const wenozn_problem* p, const double* U, double* alpha_out,
                                   int32_t* status_dev, void* stream);

/* Numerical fluxes of one sweep direction (steps of Sec. 2 and Sec. 4.3/4.4 up to, not
 * including, the flux difference): LF splitting with the given speed, Roe-averaged
 * characteristic projection (Euler), WENO-ZN reconstruction of both split parts and
 * back-projection, F^ = R (g^+ + g^-), at every interface of that direction.
 *   U     : device state [nvar][ny][nx].
 *   alpha : device, 2 doubles (8 with the per-field splitting): the LF speeds as
 *           wenozn_max_wavespeed writes them; ignored for advection, which splits with |a|
 *           (and by the local-LF and Steger-Warming splittings, which need none).
 *   dir   : 0 = x, Fout[nvar][ny][nx+1] with Fout[k][j][i] at x_{i-1/2} of row j;
 *           1 = y (2D only), Fout[nvar][ny+1][nx] with Fout[k][j][i] at y_{j-1/2};
 *           2 = both (2D only), in one launch, the form wenozn_rhs and the RK3 steps use:
 *           the x fluxes as for 0, then the y fluxes as for 1, at
 *           Fout + nvar * ny * (nx + 1).
 *   Fout  : device, overwritten; must not overlap U. */
wenozn_status wenozn_flux(const wenozn_problem* p, const double* U, const double* alpha,
                          int32_t dir, double* Fout, void* stream);

/* Semi-discrete right-hand side, Eq. (2) (1D) or its 2D form (Sec. 4.4):
 *   L = -(F^_{i+1/2} - F^_{i-1/2}) / dx  [ - (G^_{j+1/2} - G^_{j-1/2}) / dy ]
 * with global LF flux splitting (alpha of this U), Roe-averaged characteristic fields
 * (Euler) and WENO-ZN reconstruction of both split parts, ghost cells by index map.
 *   U, L : device, [nvar][ny][nx]; L is overwritten; U and L must not overlap.
 *   ws   : device workspace of ws_bytes >= wenozn_workspace_size.
 * A non-finite input state, rho <= 0, p <= 0, or a non-finite value of L (a stencil beyond
 * the reconstruction's range) sets WENOZN_ENONFINITE in the workspace status word. */
wenozn_status wenozn_rhs(const wenozn_problem* p, const double* U, double* L, void* ws,
                         size_t ws_bytes, void* stream);

/* wenozn_rhs without a workspace, for callers that cannot allocate device memory (code
 * running where cudaMalloc is unavailable or not allowed, e.g. inside a plug-in or callback
 * that must not allocate, or under a fully reserved memory pool).  The paper has no
 * counterpart: this is a property of the library, not of the scheme.
 *   U, L : device, [nvar][ny][nx]; L is overwritten; same result as wenozn_rhs.
 * Scratch comes from one 8 MiB array in the library's device memory, held on every GPU that
 * loads the library until the process exits.  Problems that need more (2D Euler beyond about
 * 131,000 cells, 1D Euler beyond about 349,000, advection beyond about 1,048,000) return
 * WENOZN_ENOMEM_WS.  Every call looks up the array's address on the current device
 * (cudaGetSymbolAddress, which allocates nothing), so it stays valid across a device reset;
 * the first call on a device also loads the library's device code there and should come
 * before any stream capture on that device.  All calls share the array and each clears what
 * must start at zero; calls whose GPU work overlaps (unordered streams) race and give wrong
 * results.  Device-detected conditions (non-finite values, rho <= 0, p <= 0) are not
 * reported, neither here nor through wenozn_last_error.  Allocates nothing. */
wenozn_status wenozn_rhs_noalloc(const wenozn_problem* p, const double* U, double* L, void* stream);

/* One third-order TVD Runge-Kutta step (Shu & Osher, cited in Sec. 4), in place:
 *   U1 = Un + dt L(Un);  U2 = 3/4 Un + 1/4 (U1 + dt L(U1));  Un+1 = 1/3 Un + 2/3 (U2 + dt L(U2)).
 *   U           : device state, advanced in place.
 *   dt          : > 0 fixed step; <= 0 CFL step computed on the device from Un
 *                 (1D: cfl dx / max(|u|+c); 2D: cfl dtx dty / (dtx + dty); advection:
 *                 cfl dx / |a|).
 *   t_remaining : > 0 clips the step to it (land on a final time); <= 0 no clipping.
 *   dt_out      : host pointer or NULL.  Non-NULL: the step taken is copied back and the
 *                 stream is synchronised.  NULL: nothing synchronises.
 *   ws          : device workspace (see wenozn_workspace_size); the step taken is also
 *                 left in it (wenozn_workspace_dt). */
wenozn_status wenozn_rk3_step(const wenozn_problem* p, double* U, double dt, double t_remaining,
                              double* dt_out, void* ws, size_t ws_bytes, void* stream);

/* wenozn_rk3_step on a state held in host memory, in one call: U_host_in is copied to the
 * device buffer U_dev, advanced by one step exactly as wenozn_rk3_step advances it (the same
 * dt, t_remaining and dt_out conventions), and copied back to U_host_out, all enqueued on
 * `stream` (cudaMemcpyAsync; with pinned host buffers the copies are asynchronous and overlap
 * work on other streams).  Alternating two streams, each with its own device buffer and
 * workspace, overlaps one step's copies with another's computation.
 *   U_host_in, U_host_out : host, [nvar][ny][nx]; they may be the same buffer.
 *   U_dev                 : device, [nvar][ny][nx], caller-owned staging buffer.
 * Allocates nothing. */
wenozn_status wenozn_rk3_step_host(const wenozn_problem* p, const double* U_host_in, double* U_host_out,
                                   double* U_dev, double dt, double t_remaining, double* dt_out, void* ws,
                                   size_t ws_bytes, void* stream);

/* A stream of `count` independent host-resident states, each advanced by one SSP-RK3 step
 * (fixed dt > 0, or its CFL step for dt <= 0) as wenozn_rk3_step would, in one call:
 * state k is copied from U_host_in[k] to the staging buffer U_dev0 (k even) or U_dev1 (k
 * odd) on upload_stream, stepped on `stream` and copied to U_host_out[k] on
 * download_stream, so that with pinned host buffers the copies of states k - 1 and k + 1
 * overlap the step of state k.  The call's work starts after the work already enqueued on
 * `stream`, and `stream` resumes only after its last copy: to the caller the call behaves
 * as one operation on `stream`.  A NULL copy stream means `stream` itself (no overlap).
 *   U_host_in, U_host_out : host arrays of `count` pointers to host [nvar][ny][nx] states
 *                           (the same pointer may repeat; an output may equal its input).
 *   U_dev0, U_dev1        : device, two distinct [nvar][ny][nx] staging buffers.
 *   ws                    : one workspace (the steps run one after another on `stream`).
 * The call creates its own ordering events and releases them before returning; it
 * allocates no memory and does not synchronise. */
wenozn_status wenozn_rk3_stream_host(const wenozn_problem* p, int64_t count, const double* const* U_host_in,
                                     double* const* U_host_out, double* U_dev0, double* U_dev1, double dt, void* ws,
                                     size_t ws_bytes, void* stream, void* upload_stream, void* download_stream);

/* The CFL step of the state U (device, [nvar][ny][nx]): the step wenozn_rk3_step takes with
 * dt <= 0 (1D: cfl dx / max(|u|+c), Sec. 4.3; 2D: cfl dtx dty / (dtx + dty) with
 * dtx = dx / max(|u|+c), dty = dy / max(|v|+c), Sec. 4.4; advection: cfl dx / |a|), from
 * the LF speeds evaluated on the device in the same IEEE operation order, so bit for bit the
 * step that call would take.  Left in the workspace's step word (wenozn_workspace_dt); when
 * the host pointer dt_out is non-NULL it is copied there and the stream is synchronised.  A
 * non-finite state, rho <= 0 or p <= 0 sets WENOZN_ENONFINITE in the status word. */
wenozn_status wenozn_cfl_dt(const wenozn_problem* p, const double* U, double* dt_out, void* ws, size_t ws_bytes,
                            void* stream);

/* nsteps SSP-RK3 steps of U in place, each with the fixed step dt > 0 or, for dt <= 0, its
 * CFL step; the same results as nsteps calls of wenozn_rk3_step, bit for bit.  The LF speeds
 * of each new state come from the last stage's update (which evaluates them anyway), so the
 * sequence needs one reduction at the start and no memset; it does not synchronise and can
 * be captured in a CUDA graph. */
wenozn_status wenozn_rk3_run(const wenozn_problem* p, double* U, int64_t nsteps, double dt, void* ws,
                             size_t ws_bytes, void* stream);

/* One SSP-RK3 step with the fixed step dt > 0, out of place, keeping what its reverse
 * (wenozn_rk3_step_vjp_stages) needs:
 *   U       : device, [nvar][ny][nx], the state U^n (read only);
 *   U_next  : device, same shape, receives U^{n+1};
 *   U1, U2  : device, same shape, receive the stage inputs U^(1), U^(2);
 *   alphas  : device, 3 doubles, receive the LF speeds of U^n, U^(1), U^(2) (x direction).
 * The five state arrays must be pairwise distinct (EINVAL otherwise).  Results equal those
 * of wenozn_rk3_step with the same dt bit for bit. */
wenozn_status wenozn_rk3_step_keep(const wenozn_problem* p, const double* U, double* U_next, double dt,
                                   double* U1, double* U2, double* alphas, void* ws, size_t ws_bytes,
                                   void* stream);

/* Device address of the FP64 time step the last wenozn_rk3_step on this workspace took. */
const double* wenozn_workspace_dt(const void* ws);

/* Synchronises `stream`, copies the workspace status word into *status (0 = clean, else
 * an OR of WENOZN_ENONFINITE / WENOZN_ETIMEOUT bits as (1 << code)) and, when `clear` is
 * non-zero, resets it. */
wenozn_status wenozn_workspace_status(void* ws, int32_t* status, int32_t clear, void* stream);

/* Synchronises `stream` and returns in *device_status the device status bits (as
 * wenozn_workspace_status reports them) raised in the control block that the most recent
 * stepping call on `stream` used (wenozn_rhs, wenozn_rk3_step, wenozn_rk3_run,
 * wenozn_rk3_step_keep, wenozn_rhs_vjp, wenozn_rk3_step_vjp, wenozn_batch_rk3_step), then
 * clears them; 0 when nothing ran on the stream.  That workspace must still be allocated. */
wenozn_status wenozn_last_error(void* stream, int32_t* device_status);

/* ---------------------------------------------------------------------------------------
 * Discrete adjoint of the 1D systems (advection and 1D Euler; 2D returns WENOZN_EINVAL).
 * Vector-Jacobian products of the scheme as implemented, with these conventions at its
 * non-smooth points: the global LF speed alpha = max_i(|u_i| + c_i) is differentiated
 * through its argmax cell (the lowest index on ties), d|x|/dx = 0 at x = 0 (in |u| and in
 * tau5 = |IS_0 - IS_2| of Eq. (tau)), and the time step of an RK3 step is a fixed input.
 * The adjoint kernels evaluate the weights without the rescaled fallback: their products
 * are exact for stencil differences between about 1e-100 and 1e25 in magnitude (with the
 * default eps = 1e-40), which covers physical Euler states by a wide margin.
 * --------------------------------------------------------------------------------------- */

/* Workspace bytes of wenozn_rhs_vjp / wenozn_rk3_step_vjp: the forward workspace of
 * wenozn_workspace_size followed by per-interface cotangent contributions (advection: 12
 * doubles per interface) or five correction records (Euler: about 4 doubles per 27 cells
 * each: the per-block sums and boundary terms one VJP launch leaves to the launches that read
 * its output), control words and two state-sized cotangent vectors.  A workspace of this
 * size also serves wenozn_rhs and wenozn_rk3_step.  Calls sharing a workspace must not run
 * concurrently. */
wenozn_status wenozn_vjp_workspace_size(const wenozn_problem* p, size_t* bytes);

/* out = J(U)^T lam with J the Jacobian of the RHS of Eq. (2) (LF splitting, Roe-averaged
 * characteristic fields, WENO-ZN), including the dependence through alpha.
 *   U, lam, out : device, [nvar][nx]; out must not overlap U or lam.  Deterministic. */
wenozn_status wenozn_rhs_vjp(const wenozn_problem* p, const double* U, const double* lam, double* out,
                             void* ws, size_t ws_bytes, void* stream);

/* Reverse of one SSP-RK3 step with the fixed step dt > 0 (the forward step being
 * wenozn_rk3_step(p, U, dt, 0, ...)): on entry lam is the cotangent of U^{n+1}, on exit the
 * cotangent of U^n = U.  The stage inputs U^(1), U^(2) are recomputed from U inside. */
wenozn_status wenozn_rk3_step_vjp(const wenozn_problem* p, const double* U, double dt, double* lam, void* ws,
                                  size_t ws_bytes, void* stream);

/* The same reverse step given the forward step's stage inputs, so nothing is recomputed:
 *   U, U1, U2 : device, the inputs U^n, U^(1), U^(2) of the three RK stages;
 *   alphas    : device, 3 doubles, the LF speeds of U^n, U^(1), U^(2) (as the forward step
 *               computed them; see wenozn_workspace_stages);
 *   lam       : cotangent of U^{n+1} on entry, of U^n on exit (must not overlap the stages). */
wenozn_status wenozn_rk3_step_vjp_stages(const wenozn_problem* p, const double* U, const double* U1,
                                         const double* U2, const double* alphas, double dt, double* lam,
                                         void* ws, size_t ws_bytes, void* stream);

/* A segment of nsteps fixed steps dt > 0 that keeps what its reverse needs, in one call:
 *   X      : device, [nsteps+1][nvar][nx]; X[0] holds U^0 on entry, X[k] receives U^k;
 *   S1, S2 : device, [nsteps][nvar][nx], the stage inputs U^(1), U^(2) of every step;
 *   alphas : device, 3 nsteps + 1 doubles: alphas[3k+s] the LF speed of the stage-s input of
 *            step k, alphas[3 nsteps] that of U^nsteps (accumulated in place, no reduction
 *            kernel per step).
 * Results equal those of nsteps calls of wenozn_rk3_step_keep bit for bit.  1D systems,
 * default scheme (as the adjoint); ws is a wenozn_vjp_workspace_size workspace. */
wenozn_status wenozn_rk3_run_keep(const wenozn_problem* p, double* X, double* S1, double* S2, double* alphas,
                                  int64_t nsteps, double dt, void* ws, size_t ws_bytes, void* stream);

/* The reverse of that segment: lam (device, [nvar][nx]) holds the cotangent of U^nsteps on
 * entry and that of U^0 on exit; the nsteps reverse steps of wenozn_rk3_step_vjp_stages run
 * from the last to the first in one call. */
wenozn_status wenozn_rk3_vjp_run(const wenozn_problem* p, const double* X, const double* S1, const double* S2,
                                 const double* alphas, int64_t nsteps, double dt, double* lam, void* ws,
                                 size_t ws_bytes, void* stream);

/* Device addresses, inside the workspace, of the stage inputs U^(1), U^(2) of the last
 * wenozn_rk3_step on it and of its LF speeds (3 doubles with a stride of 2: U^n, U^(1),
 * U^(2) at alphas[0], alphas[2], alphas[4]).  Valid until the next call on the workspace. */
wenozn_status wenozn_workspace_stages(void* ws, const wenozn_problem* p, const double** U1, const double** U2,
                                      const double** alphas);

/* ---------------------------------------------------------------------------------------
 * Batched 1D Euler: B independent problems of uneven size (the 1D Euler set-up of Sec. 4.3,
 * each with its own grid), advanced together by one persistent kernel launch per RK stage.
 *
 * Layout: U[3][total] concatenated per variable; instance b occupies columns
 * offsets[b] .. offsets[b+1]-1 (offsets[0] = 0, every instance >= 1 cell).  Each instance
 * has its own spacing dx[b], its own global LF speed (max |u|+c over its cells, per RK
 * stage), its own CFL step dt_b = cfl dx_b / alpha_b from its U^n, and its own time t_b;
 * with t_final > 0 no instance steps past t_final (finished instances are left unchanged).
 * `offsets` is the same host array of B+1 int64 on every call; the library keeps no copy
 * on the host.  The step launches no memset and does not synchronise, so a sequence of
 * steps can be captured in a CUDA graph (after wenozn_batch_init).
 * --------------------------------------------------------------------------------------- */
typedef struct {
    int32_t nbatch;   /* instances B, 1 .. 2^24                                            */
    int32_t bc;       /* wenozn_bc of every instance                                       */
    int32_t shape;    /* kernel tile shape, 0 .. wenozn_batch_num_shapes()-1; -1 = the tuned
                         shape of this batch's size class if the tuner ran on one in this
                         process (wenozn_batch_tune), else the default                      */
    int32_t flags;    /* reserved, 0                                                       */
    double gamma;     /* 1.4 (Sec. 4.3)                                                     */
    double eps;       /* Eq. (new), 1e-40                                                   */
    double A;         /* Eq. (function), 10                                                 */
    double cfl;       /* 0.5                                                                */
    double t_final;   /* > 0: stop every instance there; <= 0: no limit                     */
} wenozn_batch_params;

/* Number of compiled tile shapes, and the (interfaces per tile, threads per block) of one. */
int32_t wenozn_batch_num_shapes(void);
wenozn_status wenozn_batch_shape(int32_t shape, int32_t* tile, int32_t* threads);

/* Device workspace bytes for the batch (control block, per-instance arrays, tile prefix
 * counts of every shape, two RK stage buffers of 3 x total doubles), 256-byte aligned. */
wenozn_status wenozn_batch_workspace_size(const wenozn_batch_params* bp, const int64_t* offsets,
                                          size_t* bytes);

/* Copies offsets and dx (host arrays, B+1 and B entries) into the workspace, builds the
 * tile lists, computes every instance's LF speed of U (device, [3][total]) and sets t = 0.
 * Synchronises `stream`; the host arrays may be released afterwards.  Call it before any
 * stream capture that contains wenozn_batch_rk3_step. */
wenozn_status wenozn_batch_init(const wenozn_batch_params* bp, const int64_t* offsets, const double* dx,
                                const double* U, void* ws, size_t ws_bytes, void* stream);

/* One SSP-RK3 step of every instance (Sec. 4: third-order TVD Runge-Kutta), in place:
 * three launches of the batched stage kernel, each fusing LF splitting, characteristic
 * WENO-ZN fluxes, the flux difference of Eq. (2), the stage update and the next stage's
 * per-instance LF speeds. */
wenozn_status wenozn_batch_rk3_step(const wenozn_batch_params* bp, const int64_t* offsets, double* U,
                                    void* ws, size_t ws_bytes, void* stream);

/* Autotuner: times `steps` RK3 steps (after one warm-up step) of every compiled shape on
 * this batch, stores the fastest in bp->shape and records it in a process-wide table under
 * the batch's size class (the device, bp->bc, and floor(log2) of the mean instance size and
 * of the total cell count); ms_per_step (host, num_shapes floats) or NULL receives the
 * timings.  steps = 0 takes the table's entry for this size class without timing anything
 * (ms_per_step then holds zeros), and times 2 steps per shape when there is none yet.
 * Steps of any batch of a tuned size class with bp->shape = -1 use the recorded shape.
 * U is advanced by the trial steps: tune on a copy.  Synchronises `stream` when it times. */
wenozn_status wenozn_batch_tune(wenozn_batch_params* bp, const int64_t* offsets, double* U, void* ws,
                                size_t ws_bytes, int32_t steps, float* ms_per_step, void* stream);

/* The tile shape wenozn_batch_rk3_step uses for this batch: bp->shape if >= 0, else the
 * tuning table's entry for its size class, else the default.  Host only. */
wenozn_status wenozn_batch_resolved_shape(const wenozn_batch_params* bp, const int64_t* offsets, int32_t* shape);

/* Device addresses of the per-instance time t[B], step dt[B] (of the last RK3 step) and the
 * batch's status word inside the workspace (any output pointer may be NULL). */
wenozn_status wenozn_batch_state(void* ws, int32_t nbatch, const int64_t* offsets, double** t,
                                 double** dt, int32_t** status);

/* Static description of a status code. */
const char* wenozn_status_string(wenozn_status s);

/* Library version, "major.minor.patch". */
const char* wenozn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* WENOZN_H */
