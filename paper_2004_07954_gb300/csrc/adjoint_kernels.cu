// Discrete adjoint (vector-Jacobian products) of the 1D right-hand side and of the SSP-RK3
// step, written by hand from the forward arithmetic.
//
// RHS: L_i = -(F^_{i+1/2} - F^_{i-1/2})/dx, F^ at interface j (x_{j-1/2}) depends on the six
// cells j-3 .. j+2 and on the global LF speed alpha = max_i(|u_i| + c_i).  For a cotangent
// lambda of L the interface cotangent is Fbar_j = (lambda_j - lambda_{j-1})/dx (lambda outside
// the grid is 0).  Each interface's forward quantities are recomputed and swept backwards,
// giving the cotangents of its six stencil cells' split fluxes (and, for Euler, of its
// Roe-average inputs); every cell then sums the contributions of the stencil positions that
// map to it (ghost cells included) in a fixed order and applies its own derivatives once, so
// the result is deterministic.  Advection does the two parts in two kernels with a
// contribution buffer between them, Euler in one kernel per RK stage (below).  alpha is
// differentiated through its argmax cell (the lowest index on ties); d|x|/dx is taken as 0
// at x = 0.
#include <atomic>

#include "launch.h"

namespace wz {

namespace {

// Reverse of zn_flux: given f[0..4] and the cotangent Wb of f^ = W(f), writes dW/df * Wb to
// fb[0..4] and returns W(f).
__host__ __device__ __forceinline__ double zn_vjp(const double* f, double Wb, double eps4, double kappa,
                                                  double* fb) {
    const double a = f[0], b = f[1], c = f[2], d = f[3], e = f[4];
    // the forward of zn_num_den (fast evaluation only: the adjoint is exact for stencil
    // differences between about 1e-100 and 1e25 in magnitude): first differences, second (s_k) and one-sided (t_k)
    // differences, scaled indicators b_k, weights a_k = m^2 b0 b1 b2 + (kappa d4 P)^2 prod_{j!=k} b_j,
    // W = c + N / D with the sub-stencil fluxes q_k - c from the first differences
    const double D1 = a - b, D2 = b - c, D3 = c - d, D4 = d - e;
    const double s0 = D1 - D2, s1 = D2 - D3, s2 = D3 - D4;
    const double t0 = fma(-3.0, D2, D1), t1 = D2 + D3, t2 = fma(3.0, D3, -D4);
    const double k13_3 = 13.0 / 3.0;
    const double ks0 = k13_3 * s0, ks1 = k13_3 * s1, ks2 = k13_3 * s2;
    const double b0 = fma(ks0, s0, fma(t0, t0, eps4));
    const double b1 = fma(ks1, s1, fma(t1, t1, eps4));
    const double b2 = fma(ks2, s2, fma(t2, t2, eps4));
    const double d4 = t0 + t2;
    // b0, b2 > 0 order like their bit patterns: min/max and sign(IS_0 - IS_2) (0 on ties) on
    // the integer pipe
#ifdef __CUDA_ARCH__
    const long long i0 = __double_as_longlong(b0), i2 = __double_as_longlong(b2);
#else
    const double i0 = b0, i2 = b2;
#endif
    const double mn = i0 < i2 ? b0 : b2, mx = i0 < i2 ? b2 : b0;
    const double sg = i0 > i2 ? 1.0 : (i0 < i2 ? -1.0 : 0.0);
    const double P = fma(kappa, mx - mn, kappa * eps4);
    const double m = fma(2.0, mn, -eps4);
    const double b12 = b1 * b2, b02 = b0 * b2, b01 = b0 * b1, b012 = b01 * b2;
    const double m2 = m * m;
    const double X = m2 * b012;
    const double z = d4 * P;
    const double Y = z * z;
    const double a0 = fma(Y, b12, X), a1 = fma(Y, b02, X), a2 = fma(Y, b01, X);
    const double q0 = fma(1.0 / 3.0, D1, (-5.0 / 6.0) * D2);      // q_0 - c
    const double q1n = fma(2.0, D3, D2);                             // -6 (q_1 - c)
    const double q2 = fma(-2.0, D3, 0.5 * D4);                       // 3 (q_2 - c)
    const double N = fma(a0, q0, fma(-a1, q1n, a2 * q2));
    const double D = fma(6.0, a1, fma(3.0, a2, a0));
    const double rD = rcp_nr(D);
    const double R = N * rD;
    // reverse
    const double Nb = Wb * rD, Db = -Nb * R;
    const double a0b = fma(Nb, q0, Db), a1b = fma(-Nb, q1n, 6.0 * Db), a2b = fma(Nb, q2, 3.0 * Db);
    const double q0b = Nb * a0, q1nb = -Nb * a1, q2b = Nb * a2;
    const double Xb = (a0b + a1b) + a2b;
    const double Yb = fma(a0b, b12, fma(a1b, b02, a2b * b01));
    const double XK = Xb * m2;                       // X = m^2 b0 b1 b2
    double b0b = fma(Y, fma(a1b, b2, a2b * b1), XK * b12);
    const double b1b = fma(Y, fma(a0b, b2, a2b * b0), XK * b02);
    double b2b = fma(Y, fma(a0b, b1, a1b * b0), XK * b01);
    const double mb = (Xb * b012) * (m + m);
    const double zb = (z + z) * Yb;
    const double d4b = zb * P, Pb = zb * d4;
    // P = kappa (tau + eps4), m = b0 + b2 - tau - eps4, tau = |b0 - b2|
    const double taub = fma(kappa, Pb, -mb);
    b0b = fma(sg, taub, b0b + mb);
    b2b = fma(-sg, taub, b2b + mb);
    // b_k = (13/3) s_k^2 + t_k^2 + eps4; d4 = t0 + t2
    const double s0b = (b0b + b0b) * ks0, s1b = (b1b + b1b) * ks1, s2b = (b2b + b2b) * ks2;
    const double t0b = fma(b0b + b0b, t0, d4b), t1b = (b1b + b1b) * t1, t2b = fma(b2b + b2b, t2, d4b);
    // back through the differences: s_k = D_{k+1} - D_{k+2}, t0 = D1 - 3 D2, t1 = D2 + D3,
    // t2 = 3 D3 - D4, the q's above, D_k = f_{k-1} - f_k; W depends on c also directly
    const double D1b = fma(1.0 / 3.0, q0b, s0b + t0b);
    const double D2b = fma(-5.0 / 6.0, q0b, fma(-3.0, t0b, (s1b - s0b) + t1b) + q1nb);
    const double D3b = fma(2.0, q1nb, fma(-2.0, q2b, fma(3.0, t2b, (s2b - s1b) + t1b)));
    const double D4b = fma(0.5, q2b, -(s2b + t2b));
    fb[0] = D1b;
    fb[1] = D2b - D1b;
    fb[2] = (D3b - D2b) + Wb;
    fb[3] = D4b - D3b;
    fb[4] = -D4b;
    return c + R;
}

// ---------------------------------------------------------------------------------------
// Interface VJPs.  A block takes kTI consecutive interfaces and their kCells stencil cells,
// whose split fluxes h+- (and, for Euler, u, H, sqrt(rho), 1/rho) it computes once into
// shared memory.  For Euler each interface is then handled by three threads, one per
// characteristic field k (warp k of the block): the Roe state, row k of the left and column
// k of the right eigenvectors, the projection of the stencil onto field k, both WENO-ZN
// reconstructions of that field and their reverse sweeps.  Each field leaves its projected
// stencil's cotangents, half its left-eigenvector row and its Roe-quantity cotangents in
// shared memory; the cotangents of the split fluxes are then the sums over the fields of
// row m times the projected cotangents, and the Roe quantities' the sums of the fields'.
//
// Per interface j and stencil position s = 0..5 (cell j - 3 + s) the results are
//   (hbar+_{s,m} + hbar-_{s,m}) / 2  and  (hbar+_{s,m} - hbar-_{s,m}) / 2,  m = 0..NV-1,
// and for Euler the conserved-variable cotangents of the left (cell j - 1) and right
// (cell j) Roe-average inputs.  The split flux is h+- = (F(U) +- alpha U)/2, so
// hbar+ dh+/dU + hbar- dh-/dU is J_F^T (hbar+ + hbar-)/2 + alpha (hbar+ - hbar-)/2: the
// gather applies J_F^T once per cell to the summed first part.
// ---------------------------------------------------------------------------------------
constexpr int kTI = 32;                 // interfaces per block (one warp per field)
constexpr int kCells = kTI + 5;         // their stencil cells
constexpr int kGather = 64;             // cells per advection gather block

// The Euler stage kernel's tile: TI interfaces and their TI + 5 stencil cells; WIDE: one
// thread per interface (all three fields), else one per (interface, field).
template <int TI, bool WIDE>
struct EulerSmem {
    static constexpr int NC = TI + 5;
    double U[3][NC];
    double hp[3][NC], hm[3][NC];
    double u[NC], H[NC], sq[NC], r[NC], Ep[NC];
    double red[WIDE ? 1 : 3][WIDE ? 1 : 19][WIDE ? 1 : TI];   // per field: cotangents of its projected
                                        // h+ (5) and h- (5), half its left-eigenvector row (3), 6 Roe
                                        // scalars (the per-field threads' exchange)
};

// ---------------------------------------------------------------------------------------
// Euler: one kernel per reverse stage.  Block b owns the cells c0 = b kOwn .. c0 + kOwn - 1
// and computes the VJPs of every interface whose stencil or Roe average touches them,
// j = c0 - 2 .. c0 + kOwn + 2 (kTI of them), so that it can gather its own cells without
// anything from other blocks; neighbouring blocks both compute the five interfaces they
// share (5/kOwn more interface work, and no second launch).  Two forms: one thread per
// (interface, characteristic field) with 32-interface tiles, which gives short lines three
// times the warps, and one thread per interface with 64-interface tiles, which does less
// work per interface and serves long lines (kWideMinCells).  What the tile cannot hold
// crosses blocks through global memory:
//   - the LF-speed cotangent: every interface is owned by one block (j in [c0, c0 + kOwn),
//     and j = n by the last block), which adds its share sum_s U_s . (hbar+ - hbar-)_s / 2
//     to the block's partial;
//   - the stencil positions outside the grid (ghost cells -3..-1 and n..n+2): the summed
//     contributions of each block's owned interfaces go to that block's slot;
// A block that needs the result of every block (the sum of the partials times the speed
// derivative at the argmax cell, and the ghost contributions mapped through J_F^T to the
// cells they stand for) cannot have it before the launch ends.  So each launch leaves those
// terms in a correction record (one of kVjpRecs, in a ring: the partials, the edge blocks'
// ghost slots, the argmax candidates' speed derivatives and the argmax word), and leaves
// the at most seven cells they touch uncorrected in its output.  The launches that read
// that output later (as the cotangent input of the next stage, or as one of the RK
// combination's terms up to three stages on) apply the pending corrections as they read:
// a block resolves a record only if one of the cells it reads is a target, which only the
// first and last blocks and the block holding the argmax cell do, and forms exactly the
// value x + add (or fma(d abar, d(|u| + c)/dU, x)) that an in-place completion would have
// stored.  The last launch of a call completes in place instead: each block fences its
// writes and takes a ticket from an atomic counter (the memory-fence pattern of the CUDA
// programming guide), and the block that finishes last applies the record to the output
// and resets the argmax word and the counter.  Every sum has a fixed order, so the result
// is deterministic and does not depend on which launches complete in place.
// ---------------------------------------------------------------------------------------
constexpr int kOwn = kTI - 5;           // cells owned by a block of the per-field kernel (the most blocks)
constexpr int kGhostSlot = 6 * 9;       // 6 ghost cells x (flux, LF, Roe) x 3 components
constexpr int kEnt = 7;                 // pending corrections of a record: 6 ghost targets + the argmax
constexpr int kTIWide = 64;             // interfaces a block of the one-thread-per-interface kernel
// Lines of at least this many cells take the one-thread-per-interface kernel (fewer FP64
// instructions: no per-field copies of the Roe state, the fields' cotangents summed in
// registers, 5 of 64 interfaces computed twice instead of 5 of 32); shorter ones need the
// per-field kernel's three times as many warps to occupy the GPU.  Measured crossover:
// 8192 cells 105 (per field) against 154 us per reverse step, 12288 cells 196 against 165.
constexpr int kWideMinCells = 10240;

template <int TI, bool WIDE>
struct StageSmem {
    EulerSmem<TI, WIDE> e;
    double cF[6][3][TI], cD[6][3][TI];     // per position s, component m, interface: flux and LF parts
    double cR[2][3][TI];                   // Roe-input cotangents (left cell, right cell)
    double sF[3][TI - 5];                  // gathered flux parts, exchanged between component threads
    double ghost[6][3][3];                 // ghost slots x (flux, LF, Roe) x component
    double red[3];
    double lamw[3][TI + 1];                // the cotangent input on the window, corrections applied
    double pcq[kVjpPend][6][3];            // input records: ghost slots summed over the edge blocks,
    double pds[kVjpPend][3];               //   the argmax cell's speed derivative,
    double pred[kVjpPend][3];              //   per-warp sums of the partials,
    double pa[kVjpPend][kEnt], pb[kVjpPend][kEnt][3];   // and their entries: x <- fma(pa, pb_m, x)
    int pcell[kVjpPend][kEnt];                           //   at cell pcell (-1: none)
    int last;                              // this block finished last
    int im;                                // the LF speed's argmax cell (completion step)
    int cand;                              // the block's lowest LF-argmax candidate cell
    int tgt[6];                            // the cells the ghost slots map to (completion step)
};

// The per-warp partial sums in warp order, ((w0 + w1) + w2)
template <int W>
__device__ __forceinline__ double warp_sum(const double* w) {
    double v = w[0];
#pragma unroll
    for (int q = 1; q < W; ++q) v += w[q];
    return v;
}

// Record layout (doubles): partials [nb], ghost slots [3 edge blocks][18], candidates'
// speed derivatives [nb][3], and abar once a later launch has summed the partials.
__host__ __device__ inline int64_t rec_ghost(int nb) { return nb; }
__host__ __device__ inline int64_t rec_dsdu(int nb) { return int64_t(nb) + 54; }
__host__ __device__ inline int64_t rec_abar(int nb) { return 4 * int64_t(nb) + 54; }
__device__ inline int edge_index(int b, int nb) { return b == 0 ? 0 : (b == nb - 1 ? 2 : 1); }

// Row m of J_F^T applied to (F0, F1, F2) at a state with momentum mom, velocity u, 1/rho = r
// and E + p = Ep: F = (m, m u + p, u (E + p)), u = m/rho, p = (gamma - 1)(E - m u/2).
__device__ __forceinline__ double jft_row_q(int m, double F0, double F1, double F2, double mom, double u,
                                            double r, double Ep, double gm1) {
    const double pb = fma(F2, u, F1);
    if (m == 2) return fma(F2, u, gm1 * pb);                                      // E bar
    const double ub = fma(F1, mom, F2 * Ep) - gm1 * 0.5 * mom * pb;
    if (m == 1) return fma(ub, r, fma(F1, u, F0) - gm1 * 0.5 * u * pb);          // m bar
    return -ub * u * r;                                                            // rho bar
}

// The same at the state (rho, mom, E).
__device__ __forceinline__ double jft_row(int m, double F0, double F1, double F2, double rho, double mom,
                                          double E, double gamma) {
    const double gm1 = gamma - 1.0;
    const double r = rcp_nr(rho), u = mom * r;
    const double p = gm1 * (E - 0.5 * mom * u);
    return jft_row_q(m, F0, F1, F2, mom, u, r, E + p, gm1);
}

// Row k of the left eigenvectors (L0, L1, L2) and column k of the right ones (1, R1, R2) at
// the Roe state (u~, H~, c, 1/c, b1 = (gamma-1)/c^2, b2 = u~^2 b1 / 2).
__device__ __forceinline__ void field_lr(int k, double ut, double Ht, double c, double rc, double b1, double b2,
                                         double& L0, double& L1, double& L2, double& R1, double& R2) {
    if (k == 0) {
        L0 = 0.5 * fma(ut, rc, b2); L1 = -0.5 * fma(b1, ut, rc); L2 = 0.5 * b1;
        R1 = ut - c; R2 = fma(-ut, c, Ht);
    } else if (k == 1) {
        L0 = 1.0 - b2; L1 = b1 * ut; L2 = -b1;
        R1 = ut; R2 = 0.5 * ut * ut;
    } else {
        L0 = 0.5 * fma(-ut, rc, b2); L1 = -0.5 * fma(b1, ut, -rc); L2 = 0.5 * b1;
        R1 = ut + c; R2 = fma(ut, c, Ht);
    }
}

// The reverse of field_lr: from the cotangents of L0..L2 (Lb) and of R1, R2 (Rb1, Rb2), those
// of b2, b1, 1/c, u~, c and H~ (q[0..5]).
__device__ __forceinline__ void field_lr_reverse(int k, const double* Lb, double Rb1, double Rb2, double ut, double c,
                                                 double rc, double b1, double* q) {
    if (k == 0) {
        q[0] = 0.5 * Lb[0]; q[1] = 0.5 * fma(-ut, Lb[1], Lb[2]); q[2] = 0.5 * fma(ut, Lb[0], -Lb[1]);
        q[3] = 0.5 * fma(rc, Lb[0], -b1 * Lb[1]) + fma(-c, Rb2, Rb1); q[4] = fma(-ut, Rb2, -Rb1); q[5] = Rb2;
    } else if (k == 1) {
        q[0] = -Lb[0]; q[1] = fma(ut, Lb[1], -Lb[2]); q[2] = 0.0;
        q[3] = fma(b1, Lb[1], fma(ut, Rb2, Rb1)); q[4] = 0.0; q[5] = 0.0;
    } else {
        q[0] = 0.5 * Lb[0]; q[1] = 0.5 * fma(-ut, Lb[1], Lb[2]); q[2] = 0.5 * fma(-ut, Lb[0], Lb[1]);
        q[3] = -0.5 * fma(rc, Lb[0], b1 * Lb[1]) + fma(c, Rb2, Rb1); q[4] = fma(ut, Rb2, Rb1); q[5] = Rb2;
    }
}

// The Roe average reversed to one of its input cells: from the cotangents of b2, b1, 1/c, u~,
// c, H~ summed over the fields (sc), those of the conserved state of the cell with velocity
// uc, enthalpy Hc, 1/rho = r, sqrt(rho) = sq and weight w (w_l or w_r):
// b2 = u~^2 b1 / 2, b1 = (gamma-1) rc^2, rc = 1/c, c = sqrt((gamma-1)(H~ - u~^2/2));
// u~ = wl uL + wr uR, H~ likewise, wl = sqrt(rhoL)/(sqrt(rhoL) + sqrt(rhoR));
// u = mom/rho, H = (gamma E - (gamma-1) mom^2/(2 rho))/rho.
__device__ __forceinline__ void roe_reverse_cell(const double* sc, double ut, double Ht, double rc, double b1,
                                                 double rS, double gm1, double gamma, double w, double uc,
                                                 double Hc, double r, double sq, double* Ub) {
    double b2b = sc[0], b1b = sc[1], rcb = sc[2], utb = sc[3], cb = sc[4], Htb = sc[5];
    utb = fma(b2b * ut, b1, utb);
    b1b = fma(b2b * 0.5 * ut, ut, b1b);
    rcb = fma(b1b * 2.0 * gm1, rc, rcb);
    cb = fma(-rcb * rc, rc, cb);
    const double cq = cb * gm1 * 0.5 * rc;
    Htb += cq;
    utb = fma(-cq, ut, utb);
    const double ub = utb * w, Hb = Htb * w;
    const double sqb = fma(utb, uc - ut, Htb * (Hc - Ht)) * rS;
    Ub[0] = fma(-uc * r, ub, fma(r * fma(gm1 * 0.5 * uc, uc, -Hc), Hb, (0.5 * sqb) * (sq * r)));
    Ub[1] = r * fma(-gm1 * uc, Hb, ub);
    Ub[2] = gamma * r * Hb;
}

template <int TI, bool WIDE>
__global__ void __launch_bounds__(WIDE ? TI : 3 * TI) vjp_stage_euler(VjpArgs a) {
    constexpr int kTI = TI, kOwn = TI - 5, kCells = TI + 5, kWin = TI + 1;   // (shadow the per-field values)
    constexpr int kThreads = WIDE ? TI : 3 * TI, kWarps = kThreads / 32;
    constexpr int kLw = (3 * kWin + kThreads - 1) / kThreads;   // rounds of the window load
    constexpr int kCand = WIDE ? kThreads - 1 : 2 * kTI;        // the thread that offers the argmax candidate
    __shared__ StageSmem<TI, WIDE> S;
    EulerSmem<TI, WIDE>& sm = S.e;
    pdl_wait();
    const int n = a.n, nb = int(gridDim.x), b = int(blockIdx.x), tid = threadIdx.x;
    const int c0 = b * kOwn, j0 = c0 - 2;        // first owned cell, first interface
    const int w0 = j0 - 1;                       // first cell of the cotangent window
    const double gm1 = a.gamma - 1.0;
    const unsigned long long abits = a.alpha_bits[0];
    const double alpha = __longlong_as_double((long long)abits), half_alpha = 0.5 * alpha;
    // the record the next launch writes is no longer read by anyone: clear its argmax word
    if (b == 0 && tid == 0) a.ctl[(a.rec_out + 1) % kVjpRecs] = 0u;
    if (tid == 0) S.cand = n;
    // loads whose results are used after the cell phase: the cotangent window, the argmax
    // words of the input records and, where a ghost target lies in the window, their ghost
    // slots
    const int lo = w0 > 0 ? w0 : 0, hi = (w0 + kWin < n ? w0 + kWin : n) - 1;     // grid cells of the window
    int tg[6];
    bool gwin = false;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        tg[q] = ghost_src(q < 3 ? q - 3 : n + q - 3, n, a.bc);
        gwin = gwin || (tg[q] >= lo && tg[q] <= hi);
    }
    double lw[kLw];
#pragma unroll
    for (int t = 0; t < kLw; ++t) {
        const int q = tid + t * kThreads, m = q / kWin, g = w0 + q % kWin;
        lw[t] = q < 3 * kWin && g >= 0 && g < n ? a.lam[int64_t(m) * n + g] : 0.0;
    }
    // the input records' argmax words (uniform loads); where the argmax cell lies in the
    // window, its speed derivative and abar: the cotangent input's record sums its partials
    // (the first 4 x 96 loaded now, used after the cell phase), the others were summed by
    // the launch that read them as its cotangent input, which left abar in the record
    int imp[kVjpPend];
    bool need = false;
#pragma unroll
    for (int p = 0; p < kVjpPend; ++p) {
        const unsigned key = a.prec[p] >= 0 ? __ldcg(a.ctl + a.prec[p]) : 0u;
        imp[p] = key ? int(~key) : -1;
        need = need || (a.prec[p] >= 0 && (gwin || (imp[p] >= lo && imp[p] <= hi)));
    }
    double gsl[kVjpPend][3], pv[4] = {0.0, 0.0, 0.0, 0.0}, ds[kVjpPend], abc[kVjpPend];
#pragma unroll
    for (int p = 0; p < kVjpPend; ++p) {
        gsl[p][0] = gsl[p][1] = gsl[p][2] = 0.0;
        ds[p] = abc[p] = 0.0;
        if (a.prec[p] < 0) continue;
        const double* R = a.rec + a.prec[p] * a.rec_stride;
        if (gwin && tid < 18) {
            gsl[p][0] = __ldcg(R + rec_ghost(nb) + tid);
            if (nb >= 3) gsl[p][1] = __ldcg(R + rec_ghost(nb) + 18 + tid);
            if (nb >= 2) gsl[p][2] = __ldcg(R + rec_ghost(nb) + 36 + tid);
        }
        if (imp[p] >= lo && imp[p] <= hi) {
            if (p == a.lam_slot) {
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    if (tid + r * kThreads < nb) pv[r] = __ldcg(R + tid + r * kThreads);
            } else {
                abc[p] = __ldcg(R + rec_abar(nb));
            }
            if (tid >= 18 && tid < 21) ds[p] = __ldcg(R + rec_dsdu(nb) + int64_t(imp[p] / kOwn) * 3 + tid - 18);
        }
    }
    __syncthreads();
    for (int c = tid; c < kCells; c += kThreads) {
        const int g = j0 - 3 + c;
        const int src = ghost_src(g, n, a.bc);
        double s[3];
        for (int m = 0; m < 3; ++m) {
            s[m] = a.U[int64_t(m) * n + src];
            sm.U[m][c] = s[m];
        }
        const double rs = rsqrt(s[0]), r = rs * rs;   // 1/sqrt(rho) and 1/rho, as the forward cell phase
        const double u = s[1] * r;
        const double p = gm1 * (s[2] - 0.5 * s[1] * u);
        const double Ep = s[2] + p;
        const double F[3] = {s[1], fma(s[1], u, p), u * Ep};
        for (int m = 0; m < 3; ++m) {
            const double hF = 0.5 * F[m];
            sm.hp[m][c] = fma(half_alpha, s[m], hF);
            sm.hm[m][c] = fma(-half_alpha, s[m], hF);
        }
        sm.u[c] = u;
        sm.H[c] = Ep * r;
        sm.Ep[c] = Ep;
        sm.sq[c] = s[0] * rs;
        sm.r[c] = r;
        if (g == src && c >= 5 && c < 5 + kOwn) {   // an owned grid cell: is it the LF argmax?
            double sx, sy;
            wave_speeds<3>(s, a.gamma, sx, sy);
            if ((unsigned long long)__double_as_longlong(sx) == abits) atomicMin(&S.cand, g);
        }
    }
#pragma unroll
    for (int t = 0; t < kLw; ++t) {
        const int q = tid + t * kThreads;
        if (q < 3 * kWin) S.lamw[q / kWin][q % kWin] = lw[t];
    }
    if (need) {
        // the pending records' inputs: ghost slots summed over the edge blocks, and abar =
        // the partials summed in block order (strided runs, then the warps)
        const int kw = tid / 32;
#pragma unroll
        for (int p = 0; p < kVjpPend; ++p) {
            if (a.prec[p] < 0) continue;
            if (gwin && tid < 18) S.pcq[p][tid / 3][tid % 3] = (gsl[p][0] + gsl[p][1]) + gsl[p][2];
            if (imp[p] >= lo && imp[p] <= hi) {
                if (p == a.lam_slot) {
                    double v = 0.0;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (tid + r * kThreads < nb) v += pv[r];
                    const double* R = a.rec + a.prec[p] * a.rec_stride;
                    for (int q = tid + 4 * kThreads; q < nb; q += kThreads) v += __ldcg(R + q);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                    if ((tid & 31) == 0) S.pred[p][kw] = v;
                } else if (tid == 0) {
                    S.pred[p][0] = abc[p];
                }
                if (tid >= 18 && tid < 21) S.pds[p][tid - 18] = ds[p];
            }
        }
    }
    __syncthreads();
    // the block's lowest candidate: offered for the global argmax (the lowest index on ties),
    // with d(|u| + c)/dU of its state left in the record (|x|' = 0 at 0)
    if (tid == kCand && S.cand < n) {
        const int lc = S.cand - j0 + 3;
        atomicMax(&a.ctl[a.rec_out], ~unsigned(S.cand));
        const double rho = sm.U[0][lc], mom = sm.U[1][lc], E = sm.U[2][lc];
        const double r = rcp_nr(rho), u = mom * r;
        const double p = gm1 * (E - 0.5 * mom * u);
        const double c2 = a.gamma * p * r, rcs = rsqrt(c2);
        const double sg = u > 0.0 ? 1.0 : (u < 0.0 ? -1.0 : 0.0);
        const double kk = 0.5 * a.gamma * r * rcs;                  // gamma / (2 c rho)
        double* slot = a.rec + a.rec_out * a.rec_stride + rec_dsdu(nb) + int64_t(b) * 3;
        slot[0] = fma(sg, -u * r, kk * fma(gm1 * 0.5 * u, u, -p * r));
        slot[1] = fma(sg, r, -kk * gm1 * u);
        slot[2] = kk * gm1;
    }

    const int k = WIDE ? 0 : tid / kTI, i = WIDE ? tid : tid % kTI, j = j0 + i;
    // ---- the corrections pending on the inputs (block-uniform branches) ------------------
    if (tid < kVjpPend * kEnt * 3) {
        // entry e of record p, component mm: e < 6 the first ghost slot of a target cell in the
        // window (its slots summed in slot order, plus the LF-speed term if the cell is also
        // the argmax), e = 6 the argmax cell if it is no ghost target; the cotangent input's
        // entries are applied to the window at once (distinct cells: no two threads meet)
        const int p = tid / (kEnt * 3), e = (tid / 3) % kEnt, mm = tid % 3;
        int cell = -1;
        if (need && a.prec[p] >= 0) {
            const int im = p == 0 ? imp[0] : (p == 1 ? imp[1] : imp[2]);
            const bool im_in = im >= lo && im <= hi;
            double abar = 0.0;
            if (im_in) abar = p == a.lam_slot ? warp_sum<kWarps>(S.pred[p]) : S.pred[p][0];
            const double dabar = a.rec_d[a.prec[p]] * abar;
            if (im_in && p == a.lam_slot && e == 0 && mm == 0 && im / kOwn == b)
                a.rec[a.prec[p] * a.rec_stride + rec_abar(nb)] = abar;      // for the later readers (one writer: the owner of im)
            double pa = 1.0, pb = 0.0;
            if (e < 6) {
                int t = -1;
                bool first = true;
                double add = 0.0;
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    if (r == e) t = tg[r];
                }
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    if (r < e && tg[r] == t) first = false;
                    if (r >= e && tg[r] == t) add += S.pcq[p][r][mm];
                }
                if (first && t >= lo && t <= hi) {
                    cell = t;
                    pb = t == im ? fma(dabar, S.pds[p][mm], add) : add;
                }
            } else {
                bool im_ghost = false;
#pragma unroll
                for (int r = 0; r < 6; ++r) im_ghost = im_ghost || tg[r] == im;
                if (im_in && !im_ghost) {
                    cell = im;
                    pa = dabar;
                    pb = S.pds[p][mm];
                }
            }
            if (cell >= 0) {
                S.pa[p][e] = pa;
                S.pb[p][e][mm] = pb;
                if (p == a.lam_slot) {
                    double& x = S.lamw[mm][cell - w0];
                    x = fma(pa, pb, x);
                }
            }
        }
        if (mm == 0) S.pcell[p][e] = cell;
    }
    if (need) __syncthreads();
    const bool live = j >= 0 && j <= n;
    const bool owned = live && ((j >= c0 && j < c0 + kOwn) || (j == n && b == nb - 1));
    const int cl = i + 2, cr = i + 3;            // cells j-1, j
    double ut = 0, Ht = 0, c = 0, rc = 0, b1 = 0, b2 = 0, wl = 0, wr = 0, rS = 0;
    double Fb[3] = {0.0, 0.0, 0.0};
    if (live) {
        // Roe state (R[0][k] = 1) and the cotangents of the interface flux
        const double sl = sm.sq[cl], sr = sm.sq[cr];
        rS = rcp_nr(sl + sr);
        wl = sl * rS;
        wr = sr * rS;
        ut = fma(wl, sm.u[cl], wr * sm.u[cr]);
        Ht = fma(wl, sm.H[cl], wr * sm.H[cr]);
        const double c2 = gm1 * fma(-0.5 * ut, ut, Ht);
        rc = rsqrt(c2);
        c = c2 * rc;
        b1 = gm1 * rc * rc;
        b2 = 0.5 * ut * ut * b1;
        for (int m = 0; m < 3; ++m) Fb[m] = (S.lamw[m][i + 1] - S.lamw[m][i]) * a.rdx;   // cells j, j - 1
    }
    double ab = 0.0;
    if constexpr (!WIDE) {
        // one thread per (interface, field k): the field's projection, both reconstructions
        // and their reverse; the fields' results meet in shared memory
        if (live) {
            double L0, L1, L2, R1, R2;
            field_lr(k, ut, Ht, c, rc, b1, b2, L0, L1, L2, R1, R2);
            double fp[5], fm[5], fpb[5], fmb[5];
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                fp[s] = fma(L2, sm.hp[2][i + s], fma(L1, sm.hp[1][i + s], L0 * sm.hp[0][i + s]));
                fm[4 - s] = fma(L2, sm.hm[2][i + s + 1], fma(L1, sm.hm[1][i + s + 1], L0 * sm.hm[0][i + s + 1]));
            }
            const double ghb = fma(R2, Fb[2], fma(R1, Fb[1], Fb[0]));
            const double gh = zn_vjp(fp, ghb, a.eps4, a.kappa, fpb) +
                              zn_vjp(fm, ghb, a.eps4, a.kappa, fmb);
            double Lb[3] = {0, 0, 0};
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const double gpb = fpb[s], gmb = fmb[4 - s];     // cotangents of the projected h+_s, h-_{s+1}
#pragma unroll
                for (int m = 0; m < 3; ++m) Lb[m] = fma(gpb, sm.hp[m][i + s], fma(gmb, sm.hm[m][i + s + 1], Lb[m]));
                sm.red[k][s][i] = gpb;
                sm.red[k][5 + s][i] = gmb;
            }
            sm.red[k][10][i] = 0.5 * L0; sm.red[k][11][i] = 0.5 * L1; sm.red[k][12][i] = 0.5 * L2;
            double q[6];
            field_lr_reverse(k, Lb, Fb[1] * gh, Fb[2] * gh, ut, c, rc, b1, q);
#pragma unroll
            for (int t = 0; t < 6; ++t) sm.red[k][13 + t][i] = q[t];
        }
        __syncthreads();
        // stencil positions 2k, 2k+1: the cotangents of h+- there, (hbar+ +- hbar-)/2 summed over
        // the three fields (row m of each field's left eigenvector times its projected cotangent),
        // and, for an owned interface, its share sum_s U_s . (hbar+ - hbar-)_s / 2 of the
        // LF-speed cotangent
        double hL[3][3];
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int m = 0; m < 3; ++m) hL[f][m] = live ? sm.red[f][10 + m][i] : 0.0;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int s = 2 * k + t;
            double gp[3] = {0.0, 0.0, 0.0}, gm[3] = {0.0, 0.0, 0.0};
            if (live) {
                if (s <= 4)
#pragma unroll
                    for (int f = 0; f < 3; ++f) gp[f] = sm.red[f][s][i];
                if (s >= 1)
#pragma unroll
                    for (int f = 0; f < 3; ++f) gm[f] = sm.red[f][4 + s][i];
            }
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                // (position 5 has no plus-side point, position 0 no minus-side one)
                const double hpb = s <= 4 ? fma(gp[2], hL[2][m], fma(gp[1], hL[1][m], gp[0] * hL[0][m])) : 0.0;
                const double hmb = s >= 1 ? fma(gm[2], hL[2][m], fma(gm[1], hL[1][m], gm[0] * hL[0][m])) : 0.0;
                const double sumF = hpb + hmb, dh = hpb - hmb;
                if (owned) ab = fma(sm.U[m][i + s], dh, ab);
                S.cF[s][m][i] = sumF;
                S.cD[s][m][i] = dh;
            }
        }
        if (k > 0) {
            // the Roe average reversed: warp 1 gives the left cell, warp 2 the right
            double Ub[3] = {0.0, 0.0, 0.0};
            if (live) {
                double sc[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) sc[q] = (sm.red[0][13 + q][i] + sm.red[1][13 + q][i]) + sm.red[2][13 + q][i];
                const int cc = k == 1 ? cl : cr;
                roe_reverse_cell(sc, ut, Ht, rc, b1, rS, gm1, a.gamma, k == 1 ? wl : wr, sm.u[cc], sm.H[cc], sm.r[cc],
                                 sm.sq[cc], Ub);
            }
            for (int m = 0; m < 3; ++m) S.cR[k - 1][m][i] = Ub[m];
        }
    } else {
        // one thread per interface: the three fields in turn, their cotangents summed in
        // registers in the same order as the per-field threads sum them in shared memory
        double hpb[5][3], hmb[5][3];           // halved cotangents of h+ at cells i+s, of h- at cells i+s+1
        double sc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int m = 0; m < 3; ++m) hpb[s][m] = hmb[s][m] = 0.0;
        if (live) {
#pragma unroll 1
            for (int kf = 0; kf < 3; ++kf) {
                double L0, L1, L2, R1, R2;
                field_lr(kf, ut, Ht, c, rc, b1, b2, L0, L1, L2, R1, R2);
                double fp[5], fm[5], fpb[5], fmb[5];
#pragma unroll
                for (int s = 0; s < 5; ++s) {
                    fp[s] = fma(L2, sm.hp[2][i + s], fma(L1, sm.hp[1][i + s], L0 * sm.hp[0][i + s]));
                    fm[4 - s] = fma(L2, sm.hm[2][i + s + 1], fma(L1, sm.hm[1][i + s + 1], L0 * sm.hm[0][i + s + 1]));
                }
                const double ghb = fma(R2, Fb[2], fma(R1, Fb[1], Fb[0]));
                const double gh = zn_vjp(fp, ghb, a.eps4, a.kappa, fpb) +
                                  zn_vjp(fm, ghb, a.eps4, a.kappa, fmb);
                const double hL[3] = {0.5 * L0, 0.5 * L1, 0.5 * L2};
                double Lb[3] = {0, 0, 0};
#pragma unroll
                for (int s = 0; s < 5; ++s) {
                    const double gpb = fpb[s], gmb = fmb[4 - s];
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        Lb[m] = fma(gpb, sm.hp[m][i + s], fma(gmb, sm.hm[m][i + s + 1], Lb[m]));
                        hpb[s][m] = fma(gpb, hL[m], hpb[s][m]);
                        hmb[s][m] = fma(gmb, hL[m], hmb[s][m]);
                    }
                }
                double q[6];
                field_lr_reverse(kf, Lb, Fb[1] * gh, Fb[2] * gh, ut, c, rc, b1, q);
#pragma unroll
                for (int t = 0; t < 6; ++t) sc[t] += q[t];
            }
        }
        // stencil positions 0..5, as above
#pragma unroll
        for (int s = 0; s < 6; ++s)
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const double hp = s <= 4 ? hpb[s][m] : 0.0, hm = s >= 1 ? hmb[s - 1][m] : 0.0;
                const double sumF = hp + hm, dh = hp - hm;
                if (owned) ab = fma(sm.U[m][i + s], dh, ab);
                S.cF[s][m][i] = sumF;
                S.cD[s][m][i] = dh;
            }
        // the Roe average reversed to both input cells
        double Ul[3] = {0.0, 0.0, 0.0}, Ur[3] = {0.0, 0.0, 0.0};
        if (live) {
            roe_reverse_cell(sc, ut, Ht, rc, b1, rS, gm1, a.gamma, wl, sm.u[cl], sm.H[cl], sm.r[cl], sm.sq[cl], Ul);
            roe_reverse_cell(sc, ut, Ht, rc, b1, rS, gm1, a.gamma, wr, sm.u[cr], sm.H[cr], sm.r[cr], sm.sq[cr], Ur);
        }
        for (int m = 0; m < 3; ++m) {
            S.cR[0][m][i] = Ul[m];
            S.cR[1][m][i] = Ur[m];
        }
    }
    // deterministic per-block partial of the LF-speed cotangent (sm.red is free again)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ab += __shfl_down_sync(0xffffffffu, ab, o);
    __syncthreads();
    if ((tid & 31) == 0) S.red[tid >> 5] = ab;
    // the ghost contributions of the owned interfaces: slot q <-> cell -3 + q (q < 3) or
    // n + q - 3, summed per part (flux, LF, Roe) and component in a fixed order over the
    // positions s; only the first block and the last two can own such interfaces
    const bool edge = b == 0 || b >= nb - 2;
    if (edge && tid < kGhostSlot) {
        const int q = tid / 9, part = (tid % 9) / 3, m = tid % 3;
        const int g = q < 3 ? q - 3 : n + q - 3;
        double v = 0.0;
        for (int s = 0; s < 6; ++s) {
            const int jj = g + 3 - s, li = jj - j0;
            if (li < 0 || li >= kTI || jj < 0 || jj > n) continue;
            if (!((jj >= c0 && jj < c0 + kOwn) || (jj == n && b == nb - 1))) continue;
            if (part == 0) v += S.cF[s][m][li];
            else if (part == 1) v += S.cD[s][m][li];
            else if (s == 2) v += S.cR[0][m][li];       // left Roe input of interface jj is cell jj - 1 = g
            else if (s == 3) v += S.cR[1][m][li];       // right Roe input is cell jj = g
        }
        S.ghost[q][part][m] = v;
    }
    __syncthreads();
    double* Rout = a.rec + a.rec_out * a.rec_stride;
    if (tid == 0) Rout[b] = warp_sum<kWarps>(S.red);
    // ... and their share of the cells the ghosts map to, d (J_F^T flux + alpha LF + Roe)
    // with that cell's state: one value per slot and component
    if (edge && tid < 18) {
        const int q = tid / 3, m = tid % 3;
        const int tgt = ghost_src(q < 3 ? q - 3 : n + q - 3, n, a.bc);
        const double rho = a.U[tgt], mom = a.U[n + tgt], E = a.U[2 * int64_t(n) + tgt];
        const double jf = jft_row(m, S.ghost[q][0][0], S.ghost[q][0][1], S.ghost[q][0][2], rho, mom, E, a.gamma);
        Rout[rec_ghost(nb) + edge_index(b, nb) * 18 + tid] = a.d * (fma(alpha, S.ghost[q][1][m], jf) + S.ghost[q][2][m]);
    }
    // the gather of the owned cells: thread (m, lc) sums component m of cell c0 + lc over the
    // positions s of interfaces c0 + lc + 3 - s (fixed order), exchanges the flux parts and
    // applies row m of J_F^T
    constexpr int kGR = (3 * kOwn + kThreads - 1) / kThreads;   // rounds of the gather
    double Dsr[kGR], Rsr[kGR];
#pragma unroll
    for (int r = 0; r < kGR; ++r) {
        const int t = tid + r * kThreads, m = t / kOwn, lc = t % kOwn, cell = c0 + lc;
        const bool mine = t < 3 * kOwn && cell < n;
        double Fs = 0.0, Ds = 0.0, Rs = 0.0;
        if (mine) {
#pragma unroll
            for (int s = 0; s < 6; ++s) {
                Fs += S.cF[s][m][lc + 5 - s];
                Ds += S.cD[s][m][lc + 5 - s];
            }
            Rs = S.cR[1][m][lc + 2] + S.cR[0][m][lc + 3];
        }
        if (t < 3 * kOwn) S.sF[m][lc] = Fs;
        Dsr[r] = Ds;
        Rsr[r] = Rs;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kGR; ++r) {
        const int t = tid + r * kThreads, m = t / kOwn, lc = t % kOwn, cell = c0 + lc;
        if (!(t < 3 * kOwn && cell < n)) continue;
        const int cc = lc + 5;
        const double part = jft_row_q(m, S.sF[0][lc], S.sF[1][lc], S.sF[2][lc], sm.U[1][cc], sm.u[cc], sm.r[cc],
                                      sm.Ep[cc], gm1);
        const double Ub = fma(alpha, Dsr[r], part) + Rsr[r];
        const int64_t idx = int64_t(m) * n + cell;
        double v = a.d * Ub;
        const double* X[3] = {a.X1, a.X2, a.X3};
        const double cx[3] = {a.c1, a.c2, a.c3};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (!X[q]) continue;
            double x;
            if (a.x_slot[q] == -2) {
                x = S.lamw[m][lc + 3];                  // the cotangent input, corrected
            } else {
                x = X[q][idx];
                const int p = a.x_slot[q];
                if (p >= 0)
                    for (int e = 0; e < kEnt; ++e)
                        if (S.pcell[p][e] == cell) x = fma(S.pa[p][e], S.pb[p][e][m], x);
            }
            v = fma(cx[q], x, v);
        }
        a.out[idx] = v;
    }
    if (!a.complete) return;
    // the last launch of a call: the block that finishes last applies the record in place
    __threadfence();
    __syncthreads();
    if (tid == 0) S.last = atomicAdd(&a.ctl[kVjpRecs], 1u) == unsigned(nb - 1);
    __syncthreads();
    if (!S.last) return;
    __threadfence();
    // Everything below is a few independent L2 reads and one read-modify-write per touched
    // cell: abar = the partials summed in block order (strided runs, then the warps); the
    // edge blocks' ghost corrections per slot and component; the argmax cell's d(|u|+c)/dU,
    // left by the block that owns it.
    if (tid >= 32 && tid < 38) S.tgt[tid - 32] = ghost_src(tid < 35 ? tid - 35 : n + tid - 35, n, a.bc);
    double v = 0.0;
#pragma unroll 4
    for (int q = tid; q < nb; q += kThreads) v += __ldcg(Rout + q);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) S.red[tid >> 5] = v;
    if (tid < 18) {
        const double* G = Rout + rec_ghost(nb);             // blocks 0, nb - 2, nb - 1 (where distinct)
        double cq = __ldcg(G + tid);
        if (nb >= 3) cq += __ldcg(G + 18 + tid);
        if (nb >= 2) cq += __ldcg(G + 36 + tid);
        S.ghost[tid / 3][0][tid % 3] = cq;
    } else if (tid < 21) {
        const int mm = tid - 18;
        const unsigned key = __ldcg(a.ctl + a.rec_out);
        const int im = key ? int(~key) : -1;
        S.ghost[0][1][mm] = im >= 0 ? __ldcg(Rout + rec_dsdu(nb) + int64_t(im / kOwn) * 3 + mm) : 0.0;
        if (mm == 0) S.im = im;
    }
    __syncthreads();
    // one update per touched cell and component: the first slot of each target cell sums the
    // slots with that target in slot order, plus the LF-speed term if it is also the argmax
    const double abar = warp_sum<kWarps>(S.red);
    const int im = S.im;
    if (tid < 18) {
        const int q = tid / 3, mm = tid % 3, tgt = S.tgt[q];
        bool first = true;
        for (int r = 0; r < q; ++r) first = first && S.tgt[r] != tgt;
        if (first) {
            double add = 0.0;
            for (int r = q; r < 6; ++r)
                if (S.tgt[r] == tgt) add += S.ghost[r][0][mm];
            if (tgt == im) add = fma(a.d * abar, S.ghost[0][1][mm], add);
            double* o = a.out + int64_t(mm) * n + tgt;
            *o = __ldcg(o) + add;
        }
    } else if (tid < 21 && im >= 0) {
        const int mm = tid - 18;
        bool ghost_target = false;
        for (int r = 0; r < 6; ++r) ghost_target = ghost_target || S.tgt[r] == im;
        if (!ghost_target) {
            double* o = a.out + int64_t(mm) * n + im;
            *o = fma(a.d * abar, S.ghost[0][1][mm], __ldcg(o));
        }
    }
    __syncthreads();
    if (tid == 0) {
        a.ctl[a.rec_out] = 0u;
        a.ctl[kVjpRecs] = 0u;
    }
}

__global__ void __launch_bounds__(kTI) vjp_interface_advection(VjpArgs a) {
    __shared__ double hp[kCells], hm[kCells];
    pdl_wait();
    const int n = a.n, j0 = blockIdx.x * kTI, i = threadIdx.x, j = j0 + i;
    const int64_t P = int64_t(n) + 1;
    const double alpha = fabs(a.adv_speed);
    for (int c = i; c < kCells; c += kTI) {
        const double s = a.U[ghost_src(j0 - 3 + c, n, a.bc)];
        const double f = a.adv_speed * s;
        hp[c] = 0.5 * fma(alpha, s, f);
        hm[c] = 0.5 * fma(-alpha, s, f);
    }
    __syncthreads();
    if (j > n) return;
    const double right = j < n ? a.lam[j] : 0.0, left = j > 0 ? a.lam[j - 1] : 0.0;
    const double Fb = (right - left) * a.rdx;
    double fp[5], fm[5], fpb[5], fmb[5];
    for (int s = 0; s < 5; ++s) {
        fp[s] = hp[i + s];
        fm[4 - s] = hm[i + s + 1];
    }
    zn_vjp(fp, Fb, a.eps4, a.kappa, fpb);
    zn_vjp(fm, Fb, a.eps4, a.kappa, fmb);
    for (int s = 0; s < 6; ++s) {
        const double hpb = s <= 4 ? fpb[s] : 0.0, hmb = s >= 1 ? fmb[5 - s] : 0.0;
        a.C[(2 * s) * P + j] = 0.5 * (hpb + hmb);
        a.C[(2 * s + 1) * P + j] = 0.5 * (hpb - hmb);
    }
}

// Per cell i: sum the contributions of the stencil positions that map to it (ghost cells
// included, fixed order), apply the cell's own derivatives once and write
// out_i = c1 X1_i + c2 X2_i + c3 X3_i + d (J^T lambda)_i.  Advection: f = a u, so the flux
// part takes the factor a and the LF part |a|.
__global__ void __launch_bounds__(kGather) vjp_gather_advection(VjpArgs a) {
    pdl_wait();
    const int n = a.n;
    const int64_t P = int64_t(n) + 1;
    const int i = blockIdx.x * kGather + threadIdx.x;
    if (i >= n) return;
    double Fs = 0.0, Ds = 0.0;
    if (i >= 3 && i <= n - 4) {
        // interior: the cell is stencil position s of interface i + 3 - s only
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            const int64_t j = i + 3 - s;
            Fs += a.C[(s * 2) * P + j];
            Ds += a.C[(s * 2 + 1) * P + j];
        }
    } else {
        int gs[16], ng = 0;             // stencil cells g (in -3 .. n+2) that map to i
        if (n <= 8) {
            for (int g = -3; g <= n + 2; ++g)
                if (ghost_src(g, n, a.bc) == i) gs[ng++] = g;
        } else if (a.bc == 0) {
            for (int g = i - n; g <= i + n; g += n)
                if (g >= -3 && g <= n + 2) gs[ng++] = g;
        } else {
            gs[ng++] = i;
            if (i == 0) { gs[ng++] = -1; gs[ng++] = -2; gs[ng++] = -3; }
            if (i == n - 1) { gs[ng++] = n; gs[ng++] = n + 1; gs[ng++] = n + 2; }
        }
        for (int q = 0; q < ng; ++q) {
            const int g = gs[q];
            for (int s = 0; s < 6; ++s) {
                const int j = g + 3 - s;         // interface whose stencil position s is g
                if (j < 0 || j > n) continue;
                Fs += a.C[(s * 2) * P + j];
                Ds += a.C[(s * 2 + 1) * P + j];
            }
        }
    }
    double v = a.d * fma(a.adv_speed, Fs, fabs(a.adv_speed) * Ds);
    if (a.X1) v = fma(a.c1, a.X1[i], v);
    if (a.X2) v = fma(a.c2, a.X2[i], v);
    if (a.X3) v = fma(a.c3, a.X3[i], v);
    a.out[i] = v;
}

}  // namespace

// The Euler stage kernel is FP64-bound and as fast as its busiest SM: the block scheduler
// balances it over empty SMs (two blocks per SM at the sizes where it matters), but
// launched with programmatic dependent launch its blocks become resident (and wait) while
// the previous launch drains, and would pile up on the SMs that launch leaves free first.
// An unused dynamic shared-memory reservation caps it at two blocks per SM, which keeps the
// balanced placement.  The reservation is sized per device, once.
static cudaError_t euler_interface_pad(size_t* pad) {
    static std::atomic<unsigned long long> configured{0};
    static size_t pads[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        int per_sm = 0, reserved = 0;
        e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (e != cudaSuccess) return e;
        const long budget = long(per_sm) / 2 - long(reserved) - long(sizeof(StageSmem<kTI, false>)) - 1024;
        size_t pd = budget > 0 ? size_t(budget) : 0;
        if (pd > 0) {
            e = cudaFuncSetAttribute(vjp_stage_euler<kTI, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(pd));
            if (e != cudaSuccess) return e;
        }
        pads[dev & 63] = pd;
        configured.fetch_or(bit);
    }
    *pad = pads[dev & 63];
    return cudaSuccess;
}

// one correction record of the Euler stage kernel, in doubles (a multiple of 32)
int64_t vjp_rec_stride(int n) {
    const int64_t nb = (int64_t(n) + kOwn - 1) / kOwn;
    return (rec_abar(int(nb)) + 1 + 31) / 32 * 32;
}

// per-interface contributions (advection), or the Euler stage kernel's correction records
size_t vjp_contrib_doubles(int nv, int n) {
    return nv == 1 ? size_t(n + 1) * 12 : size_t(kVjpRecs) * size_t(vjp_rec_stride(n));
}

cudaError_t launch_vjp(int system, const VjpArgs& a, cudaStream_t s) {
    if (system == 0) {
        const unsigned gi = unsigned((a.n + 1 + kTI - 1) / kTI), gc = unsigned((a.n + kGather - 1) / kGather);
        cudaError_t e = launch_pdl(vjp_interface_advection, dim3(gi), dim3(kTI), 0, s, a);
        if (e == cudaSuccess) e = launch_pdl(vjp_gather_advection, dim3(gc), dim3(kGather), 0, s, a);
        return e;
    }
    if (a.n >= kWideMinCells)
        return launch_pdl(vjp_stage_euler<kTIWide, true>, dim3(unsigned((a.n + kTIWide - 6) / (kTIWide - 5))),
                          dim3(kTIWide), 0, s, a);
    size_t pad = 0;
    cudaError_t e = euler_interface_pad(&pad);
    if (e == cudaSuccess)
        e = launch_pdl(vjp_stage_euler<kTI, false>, dim3(unsigned((a.n + kOwn - 1) / kOwn)), dim3(3 * kTI), pad, s, a);
    return e;
}

}  // namespace wz
