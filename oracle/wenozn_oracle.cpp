// WENO-ZN oracle: TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, loop-per-interface CPU restatement of the WENO-ZN finite-difference
// solver of Shen, Zhang, Li & Peng ("A novel method for constructing high accurate and
// robust WENO-Z type scheme", arXiv 2004.07954).  It exists to check the CUDA library
// against, and only the test suite, the smoke check and the benchmark's CPU-baseline leg
// may load it.  It shares no code, header, constant table or helper with the CUDA path.
//
// Every routine is written in the paper's order and notation.  No fusion, no algebraic
// rewriting, no reordering beyond what the formulas state.  Templated on the scalar type:
//   double   - the reference arithmetic for parity tests,
//   Quad     - binary128 (x86: __float128, aarch64: long double) for the Sec. 4.1 table,
//   OpCount  - counts the algorithmic floating-point operations of one RHS evaluation.
//
// Readings where the paper is silent (each is listed with its justification in the
// project's design notes):
//   eps = 1e-40 in Eq. (new) (reproduces every digit of the Sec. 4.1 table), q = 1,
//   tau in Eq. (function) is tau5, the minus-side flux is the same formula applied to the
//   mirrored stencil, global Lax-Friedrichs splitting with one alpha per direction per RK
//   stage, Roe-averaged characteristic fields (all six stencil points projected with the
//   interface's left eigenvectors), Shu-Osher SSP-RK3, three ghost cells per side.
//
// Parity pins of this file live in the CPU test suite: the Sec. 3 coefficient table, the
// Sec. 3 worked example table, the Sec. 4.1 critical-point table, closed forms on
// polynomial and step data, the Roe property, L*J*R = diag(lambda), the RK3 stability
// polynomial, exact-solution convergence and conservation.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

#if defined(__x86_64__)
typedef __float128 Quad;
#else
typedef long double Quad;   // IEEE binary128 on aarch64
#endif

namespace orc {

// ---------------------------------------------------------------------------------------
// Operation counter (algorithmic flops: one per +, -, *, /, sqrt; comparisons apart).
// ---------------------------------------------------------------------------------------
struct OpTally { long long add = 0, mul = 0, div = 0, sqrt_ = 0, cmp = 0; };
static OpTally g_tally;

struct OpCount {
    double v;
    OpCount() : v(0) {}
    explicit OpCount(double x) : v(x) {}
};
inline OpCount operator+(OpCount a, OpCount b) { g_tally.add++; return OpCount(a.v + b.v); }
inline OpCount operator-(OpCount a, OpCount b) { g_tally.add++; return OpCount(a.v - b.v); }
inline OpCount operator*(OpCount a, OpCount b) { g_tally.mul++; return OpCount(a.v * b.v); }
inline OpCount operator/(OpCount a, OpCount b) { g_tally.div++; return OpCount(a.v / b.v); }
inline OpCount operator-(OpCount a) { return OpCount(-a.v); }
inline bool operator<(OpCount a, OpCount b) { g_tally.cmp++; return a.v < b.v; }
inline bool operator>(OpCount a, OpCount b) { g_tally.cmp++; return a.v > b.v; }
inline OpCount& operator+=(OpCount& a, OpCount b) { a = a + b; return a; }

// Exact rational constant num/den in type T (not counted as an operation).
template <class T> inline T cst(int num, int den) { return T(num) / T(den); }
template <> inline OpCount cst<OpCount>(int num, int den) { return OpCount(double(num) / double(den)); }

template <class T> inline T tabs(T x) { return x < T(0) ? -x : x; }
template <class T> inline T tmax(T a, T b) { return a < b ? b : a; }
inline double tsqrt(double x) { return std::sqrt(x); }
inline OpCount tsqrt(OpCount x) { g_tally.sqrt_++; return OpCount(std::sqrt(x.v)); }
template <class T> inline double tod(T x) { return double(x); }
inline double tod(OpCount x) { return x.v; }

// ---------------------------------------------------------------------------------------
// Forward-mode dual number (value, derivative along one direction): running the solver on
// it gives the exact Jacobian-vector product of the discrete scheme.  Conventions at the
// scheme's non-smooth points: d|x|/dx = 0 at x = 0; a maximum passes the derivative of the
// selected argument (the first one on ties, i.e. the lowest cell index for the LF speed).
// ---------------------------------------------------------------------------------------
template <class S> inline S sqrt_of(S x);
template <> inline double sqrt_of<double>(double x) { return std::sqrt(x); }
// binary128 square root: two Newton steps from the double one (quadratic convergence)
template <> inline Quad sqrt_of<Quad>(Quad x) {
    if (!(x > 0)) return Quad(0);
    Quad r = Quad(std::sqrt(double(x)));
    r = (r + x / r) / Quad(2);
    r = (r + x / r) / Quad(2);
    return r;
}

template <class S> struct DualT {
    S v, d;
    DualT() : v(0), d(0) {}
    explicit DualT(S x) : v(x), d(0) {}
    DualT(S x, S dx) : v(x), d(dx) {}
};
template <class S> inline DualT<S> operator+(DualT<S> a, DualT<S> b) { return DualT<S>(a.v + b.v, a.d + b.d); }
template <class S> inline DualT<S> operator-(DualT<S> a, DualT<S> b) { return DualT<S>(a.v - b.v, a.d - b.d); }
template <class S> inline DualT<S> operator*(DualT<S> a, DualT<S> b) {
    return DualT<S>(a.v * b.v, a.d * b.v + a.v * b.d);
}
template <class S> inline DualT<S> operator/(DualT<S> a, DualT<S> b) {
    return DualT<S>(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
template <class S> inline DualT<S> operator-(DualT<S> a) { return DualT<S>(-a.v, -a.d); }
template <class S> inline bool operator<(DualT<S> a, DualT<S> b) { return a.v < b.v; }
template <class S> inline bool operator>(DualT<S> a, DualT<S> b) { return a.v > b.v; }
template <class S> inline DualT<S>& operator+=(DualT<S>& a, DualT<S> b) { a = a + b; return a; }
template <class S> inline DualT<S> tsqrt(DualT<S> x) {
    const S r = sqrt_of<S>(x.v);
    return DualT<S>(r, x.d / (S(2) * r));
}
template <class S> inline double tod(DualT<S> x) { return double(x.v); }
template <class S> inline DualT<S> tabs_dual(DualT<S> x) {
    if (x.v < S(0)) return -x;
    if (x.v > S(0)) return x;
    return DualT<S>(S(0), S(0));
}
typedef DualT<double> Dual;
typedef DualT<Quad> DualQ;
template <> inline Dual tabs<Dual>(Dual x) { return tabs_dual(x); }
template <> inline DualQ tabs<DualQ>(DualQ x) { return tabs_dual(x); }

// ---------------------------------------------------------------------------------------
// Sec. 2.1 / Sec. 3: one fifth-order reconstruction f^+_{i+1/2} from (f_{i-2},...,f_{i+2}).
// ---------------------------------------------------------------------------------------
enum WeightKind { W_ZN = 0, W_Z = 1, W_LINEAR = 2, W_JS = 3 };

template <class T> struct WenoParts {
    T q[3], IS[3], tau5, tau8, C, alpha[3], omega[3], fhat;
};

template <class T>
WenoParts<T> weno5(const T f[5], T eps, T A, int kind) {
    WenoParts<T> r;
    const T fm2 = f[0], fm1 = f[1], f0 = f[2], fp1 = f[3], fp2 = f[4];
    // Eq. (4): third-order fluxes on the sub-stencils S_k = (i+k-2, i+k-1, i+k).
    r.q[0] = cst<T>(1, 3) * fm2 - cst<T>(7, 6) * fm1 + cst<T>(11, 6) * f0;
    r.q[1] = -cst<T>(1, 6) * fm1 + cst<T>(5, 6) * f0 + cst<T>(1, 3) * fp1;
    r.q[2] = cst<T>(1, 3) * f0 + cst<T>(5, 6) * fp1 - cst<T>(1, 6) * fp2;
    // Eq. (isjiang): Jiang-Shu local smoothness indicators.
    {
        T a = fm2 - T(2) * fm1 + f0, b = fm2 - T(4) * fm1 + T(3) * f0;
        r.IS[0] = cst<T>(13, 12) * a * a + cst<T>(1, 4) * b * b;
    }
    {
        T a = fm1 - T(2) * f0 + fp1, b = fm1 - fp1;
        r.IS[1] = cst<T>(13, 12) * a * a + cst<T>(1, 4) * b * b;
    }
    {
        // the mirror image of IS_0's one-sided difference, (f_{i+2} - 4 f_{i+1}) + 3 f_i: like
        // IS_0's it is exactly zero on constant data
        T a = f0 - T(2) * fp1 + fp2, b = fp2 - T(4) * fp1 + T(3) * f0;
        r.IS[2] = cst<T>(13, 12) * a * a + cst<T>(1, 4) * b * b;
    }
    // Eq. (tau) = Eq. (tao5): tau5 = |IS_0 - IS_2|.
    r.tau5 = tabs(r.IS[0] - r.IS[2]);
    // Eq. (tau8): square of the five-point fourth difference.
    {
        // summed symmetrically, (f_{i-2} + f_{i+2}) - 4 (f_{i-1} + f_{i+1}) + 6 f_i, which is
        // exactly zero on constant data
        T d4 = (fm2 + fp2) - T(4) * (fm1 + fp1) + T(6) * f0;
        r.tau8 = d4 * d4;
    }
    // Eq. (function): C = A ((IS_0 + IS_2 - tau + eps) / (tau + eps))^2.
    {
        T ratio = (r.IS[0] + r.IS[2] - r.tau5 + eps) / (r.tau5 + eps);
        r.C = A * ratio * ratio;
    }
    const T c[3] = {cst<T>(1, 10), cst<T>(6, 10), cst<T>(3, 10)};   // Sec. 2.1 optimal weights
    for (int k = 0; k < 3; ++k) {
        if (kind == W_ZN)        // Eq. (new)
            r.alpha[k] = c[k] * (r.C + r.tau8 / (r.IS[k] + eps));
        else if (kind == W_Z)    // Eq. (15) with q = 1
            r.alpha[k] = c[k] * (T(1) + r.tau5 / (r.IS[k] + eps));
        else if (kind == W_JS)   // Sec. 2.1, the Jiang-Shu weights c_k / (IS_k + eps)^2
            r.alpha[k] = c[k] / ((r.IS[k] + eps) * (r.IS[k] + eps));
        else                     // linear fifth-order upwind scheme
            r.alpha[k] = c[k];
    }
    // Eq. (3) / (15): normalisation and the convex combination.
    T sum = r.alpha[0] + r.alpha[1] + r.alpha[2];
    for (int k = 0; k < 3; ++k) r.omega[k] = r.alpha[k] / sum;
    r.fhat = r.omega[0] * r.q[0] + r.omega[1] * r.q[1] + r.omega[2] * r.q[2];
    return r;
}

// Minus-side flux (Sec. 2, "symmetric rule about x_{i+1/2}"): the same formula applied to
// (f_{i+3}, f_{i+2}, f_{i+1}, f_i, f_{i-1}).
template <class T>
T weno5_minus(const T f_im1_to_ip3[5], T eps, T A, int kind) {
    T m[5] = {f_im1_to_ip3[4], f_im1_to_ip3[3], f_im1_to_ip3[2], f_im1_to_ip3[1], f_im1_to_ip3[0]};
    return weno5(m, eps, A, kind).fhat;
}

// ---------------------------------------------------------------------------------------
// Problem description (the oracle's own copy; it mirrors the library's fields by value).
// ---------------------------------------------------------------------------------------
struct Problem {
    int32_t system, nx, ny, bc_x, bc_y, weights;   // weights: WeightKind
    int32_t split, pad;                            // split: SplitKind
    double dx, dy, gamma, eps, A, cfl, adv_speed;
};
enum { SYS_ADV1D = 0, SYS_EULER1D = 1, SYS_EULER2D = 2 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_REFLECTIVE = 2 };
// Flux splitting: global Lax-Friedrichs with one speed per direction (the hot path), global
// LF with one speed per characteristic field, local LF with the largest |u| + c of the
// interface's six stencil cells, and Steger-Warming flux-vector splitting (Sec. 4.4).
enum SplitKind { S_LF = 0, S_LF_FIELD = 1, S_LLF = 2, S_SW = 3 };

inline int nvar_of(int system) { return system == SYS_ADV1D ? 1 : (system == SYS_EULER1D ? 3 : 4); }

// Ghost-cell index map: periodic wrap (Sec. 4.2), zero-order extrapolation (outflow), or
// the mirror image across the wall (reflective: cell -1-i for i < 0, 2n-1-i for i >= n,
// repeated, i.e. the grid continued with period 2n and mirrored in every other copy).
inline int64_t ghost_src(int64_t i, int64_t n, int bc) {
    if (bc == BC_PERIODIC) return ((i % n) + n) % n;
    if (bc == BC_REFLECTIVE) {
        const int64_t m = ((i % (2 * n)) + 2 * n) % (2 * n);
        return m < n ? m : 2 * n - 1 - m;
    }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}
// A reflective ghost that is a mirror image carries the opposite normal momentum.
inline bool ghost_mirrored(int64_t i, int64_t n, int bc) {
    if (bc != BC_REFLECTIVE) return false;
    const int64_t m = ((i % (2 * n)) + 2 * n) % (2 * n);
    return m >= n;
}

// ---------------------------------------------------------------------------------------
// Euler system along one direction (Sec. 4.3 / 4.4).  The state is written in the
// direction's frame: (rho, m_n, E) in 1D, (rho, m_n, m_t, E) in 2D, where m_n is the
// momentum normal to the interface and m_t the tangential one.  The y-sweep of the 2D
// problem uses the same formulas on (rho, rho v, rho u, E).
// ---------------------------------------------------------------------------------------
template <class T> struct Prim { T rho, un, ut, E, p; };

template <class T>
Prim<T> primitives(const T* U, int nv, T gamma) {
    Prim<T> w;
    w.rho = U[0];
    w.un = U[1] / w.rho;
    w.ut = nv == 4 ? U[2] / w.rho : T(0);
    w.E = U[nv - 1];
    T kin = nv == 4 ? cst<T>(1, 2) * w.rho * (w.un * w.un + w.ut * w.ut)
                    : cst<T>(1, 2) * w.rho * w.un * w.un;
    w.p = (gamma - T(1)) * (w.E - kin);                    // equation of state
    return w;
}
template <class T> T sound_speed(const Prim<T>& w, T gamma) { return tsqrt(gamma * w.p / w.rho); }
template <class T> T enthalpy(const Prim<T>& w) { return (w.E + w.p) / w.rho; }

// Physical flux normal to the interface, F(U) (Sec. 4.3) or its 2D form (Sec. 4.4).
template <class T>
void normal_flux(const T* U, const Prim<T>& w, int nv, T* F) {
    F[0] = U[1];
    F[1] = U[1] * w.un + w.p;
    if (nv == 4) F[2] = U[2] * w.un;
    F[nv - 1] = w.un * (w.E + w.p);
}

// Roe average of the left and right states (weights sqrt(rho)) and the eigenvectors of the
// flux Jacobian there.  R holds the right eigenvectors as columns, Lm the left ones as
// rows (Lm = R^-1).
template <class T> struct Eigen { T un, ut, H, c; T R[4][4]; T Lm[4][4]; };

template <class T>
Eigen<T> roe_eigen_from(T sl, T unl, T utl, T Hl, T sr, T unr, T utr, T Hr, int nv, T gamma) {
    Eigen<T> e;
    e.un = (sl * unl + sr * unr) / (sl + sr);
    e.ut = nv == 4 ? (sl * utl + sr * utr) / (sl + sr) : T(0);
    e.H = (sl * Hl + sr * Hr) / (sl + sr);
    T q2 = nv == 4 ? e.un * e.un + e.ut * e.ut : e.un * e.un;
    e.c = tsqrt((gamma - T(1)) * (e.H - cst<T>(1, 2) * q2));
    const T u = e.un, v = e.ut, H = e.H, c = e.c;
    const T b1 = (gamma - T(1)) / (c * c), b2 = cst<T>(1, 2) * q2 * b1;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) e.R[i][j] = e.Lm[i][j] = T(0);
    if (nv == 3) {
        // columns: lambda = u - c, u, u + c
        e.R[0][0] = T(1);      e.R[0][1] = T(1);                  e.R[0][2] = T(1);
        e.R[1][0] = u - c;     e.R[1][1] = u;                     e.R[1][2] = u + c;
        e.R[2][0] = H - u * c; e.R[2][1] = cst<T>(1, 2) * u * u;  e.R[2][2] = H + u * c;
        e.Lm[0][0] = cst<T>(1, 2) * (b2 + u / c);
        e.Lm[0][1] = -cst<T>(1, 2) * (b1 * u + T(1) / c);
        e.Lm[0][2] = cst<T>(1, 2) * b1;
        e.Lm[1][0] = T(1) - b2;
        e.Lm[1][1] = b1 * u;
        e.Lm[1][2] = -b1;
        e.Lm[2][0] = cst<T>(1, 2) * (b2 - u / c);
        e.Lm[2][1] = -cst<T>(1, 2) * (b1 * u - T(1) / c);
        e.Lm[2][2] = cst<T>(1, 2) * b1;
    } else {
        // columns: lambda = u - c, u, u (shear), u + c; state (rho, m_n, m_t, E)
        e.R[0][0] = T(1);      e.R[0][1] = T(1);                e.R[0][2] = T(0); e.R[0][3] = T(1);
        e.R[1][0] = u - c;     e.R[1][1] = u;                   e.R[1][2] = T(0); e.R[1][3] = u + c;
        e.R[2][0] = v;         e.R[2][1] = v;                   e.R[2][2] = T(1); e.R[2][3] = v;
        e.R[3][0] = H - u * c; e.R[3][1] = cst<T>(1, 2) * q2;   e.R[3][2] = v;    e.R[3][3] = H + u * c;
        e.Lm[0][0] = cst<T>(1, 2) * (b2 + u / c);
        e.Lm[0][1] = -cst<T>(1, 2) * (b1 * u + T(1) / c);
        e.Lm[0][2] = -cst<T>(1, 2) * b1 * v;
        e.Lm[0][3] = cst<T>(1, 2) * b1;
        e.Lm[1][0] = T(1) - b2;
        e.Lm[1][1] = b1 * u;
        e.Lm[1][2] = b1 * v;
        e.Lm[1][3] = -b1;
        e.Lm[2][0] = -v;
        e.Lm[2][1] = T(0);
        e.Lm[2][2] = T(1);
        e.Lm[2][3] = T(0);
        e.Lm[3][0] = cst<T>(1, 2) * (b2 - u / c);
        e.Lm[3][1] = -cst<T>(1, 2) * (b1 * u - T(1) / c);
        e.Lm[3][2] = -cst<T>(1, 2) * b1 * v;
        e.Lm[3][3] = cst<T>(1, 2) * b1;
    }
    return e;
}

template <class T>
Eigen<T> roe_eigen(const T* UL, const T* UR, int nv, T gamma) {
    Prim<T> l = primitives(UL, nv, gamma), r = primitives(UR, nv, gamma);
    return roe_eigen_from(tsqrt(l.rho), l.un, l.ut, enthalpy(l), tsqrt(r.rho), r.un, r.ut,
                          enthalpy(r), nv, gamma);
}

// Steger-Warming splitting of the flux normal to the interface (Steger & Warming 1981, the
// splitting of Sec. 4.4): with the eigenvalues l1 = u - c, l2 = u, l3 = u + c and
// l+- = (l +- |l|)/2,
//   F+- = rho/(2 gamma) ( 2(gamma-1) l2 + l1 + l3,
//                         2(gamma-1) l2 u + l1 (u - c) + l3 (u + c),
//                        [2(gamma-1) l2 v + l1 v + l3 v,]
//                         (gamma-1) l2 q^2 + l1 ((u-c)^2 + v^2)/2 + l3 ((u+c)^2 + v^2)/2
//                           + (3 - gamma)(l1 + l3) c^2 / (2 (gamma - 1)) )      (l = l+-),
// q^2 = u^2 + v^2 (v = 0 in 1D); F+ + F- = F.
template <class T>
void steger_warming(const Prim<T>& w, int nv, T gamma, int sign, T* Fs) {
    const T c = sound_speed(w, gamma);
    const T u = w.un, v = w.ut;
    const T lam[3] = {u - c, u, u + c};
    T l[3];
    for (int k = 0; k < 3; ++k) l[k] = cst<T>(1, 2) * (lam[k] + T(sign) * tabs(lam[k]));
    const T g1 = gamma - T(1);
    const T q2 = nv == 4 ? u * u + v * v : u * u;
    const T k0 = w.rho / (T(2) * gamma);
    Fs[0] = k0 * (T(2) * g1 * l[1] + l[0] + l[2]);
    Fs[1] = k0 * (T(2) * g1 * l[1] * u + l[0] * (u - c) + l[2] * (u + c));
    if (nv == 4) Fs[2] = k0 * (T(2) * g1 * l[1] * v + l[0] * v + l[2] * v);
    const T um = u - c, up = u + c;
    const T vv = nv == 4 ? v * v : T(0);
    Fs[nv - 1] = k0 * (g1 * l[1] * q2 + cst<T>(1, 2) * l[0] * (um * um + vv) + cst<T>(1, 2) * l[2] * (up * up + vv)
                       + (T(3) - gamma) * (l[0] + l[2]) * c * c / (T(2) * g1));
}

// Per-cell quantities of one padded grid line, each computed once per cell, by splitting:
//   S_LF       hp, hm = (F +- alpha U)/2 (LF splitting, Sec. 2 and Sec. 4.3);
//   S_LF_FIELD, S_LLF: hp = F, hm = U (split per field or per interface after projection),
//              and for S_LLF the cell's |u_n| + c in `speed`;
//   S_SW       hp, hm = F+, F- (Steger-Warming);
// and, for the Euler systems, the Roe-average ingredients sqrt(rho), u_n, u_t, H.
template <class T> struct LineCells {
    std::vector<T> hp, hm, srho, un, ut, H, speed;
};

// `par`: spread the cells over the OpenMP threads (a single long line; the cells are
// independent, so the results do not depend on it).
template <class T>
void line_cells(const Problem& P, const T* Ul, int64_t np, int nv, T alpha, LineCells<T>& lc, bool par = false) {
    lc.hp.resize(np * nv); lc.hm.resize(np * nv);
    if (P.system == SYS_ADV1D) {
        const T a = T(P.adv_speed);
#pragma omp parallel for schedule(static) if (par && np > 4096)
        for (int64_t p = 0; p < np; ++p) {
            T f = a * Ul[p];
            lc.hp[p] = cst<T>(1, 2) * (f + alpha * Ul[p]);
            lc.hm[p] = cst<T>(1, 2) * (f - alpha * Ul[p]);
        }
        return;
    }
    const T gamma = T(P.gamma);
    lc.srho.resize(np); lc.un.resize(np); lc.ut.resize(np); lc.H.resize(np); lc.speed.resize(np);
#pragma omp parallel for schedule(static) if (par && np > 4096)
    for (int64_t p = 0; p < np; ++p) {
        const T* U = &Ul[p * nv];
        Prim<T> w = primitives(U, nv, gamma);
        T F[4];
        normal_flux(U, w, nv, F);
        if (P.split == S_LF) {
            for (int m = 0; m < nv; ++m) {
                lc.hp[p * nv + m] = cst<T>(1, 2) * (F[m] + alpha * U[m]);
                lc.hm[p * nv + m] = cst<T>(1, 2) * (F[m] - alpha * U[m]);
            }
        } else if (P.split == S_SW) {
            steger_warming(w, nv, gamma, +1, &lc.hp[p * nv]);
            steger_warming(w, nv, gamma, -1, &lc.hm[p * nv]);
        } else {
            for (int m = 0; m < nv; ++m) {
                lc.hp[p * nv + m] = F[m];
                lc.hm[p * nv + m] = U[m];
            }
            lc.speed[p] = tabs(w.un) + sound_speed(w, gamma);
        }
        lc.srho[p] = tsqrt(w.rho);
        lc.un[p] = w.un;
        lc.ut[p] = w.ut;
        lc.H[p] = enthalpy(w);
    }
}

// Numerical flux at the interface between padded cells i and i+1 of one grid line.
// alpha_f: the per-field LF speeds of the sweep (S_LF_FIELD), indexed by eigenvalue kind
// (0: u - c, 1: u, 2: u + c).
template <class T>
void interface_flux(const Problem& P, const LineCells<T>& lc, int nv, int64_t i, T* Fhat,
                    const T* alpha_f = nullptr) {
    const T eps = T(P.eps), A = T(P.A);
    if (P.system == SYS_ADV1D) {
        // f^+ from cells i-2..i+2, f^- from the mirrored cells i+3..i-1
        Fhat[0] = weno5(&lc.hp[i - 2], eps, A, P.weights).fhat
                + weno5_minus(&lc.hm[i - 1], eps, A, P.weights);
        return;
    }
    const T gamma = T(P.gamma);
    Eigen<T> e = roe_eigen_from(lc.srho[i], lc.un[i], lc.ut[i], lc.H[i], lc.srho[i + 1],
                                lc.un[i + 1], lc.ut[i + 1], lc.H[i + 1], nv, gamma);
    // characteristic projection with the interface's left eigenvectors:
    // g+ of cells i-2..i+2 and g- of cells i-1..i+3
    T gp[5][4], gm[5][4];
    if (P.split == S_LF || P.split == S_SW) {
        for (int s = 0; s < 5; ++s)
            for (int k = 0; k < nv; ++k) {
                T accp = T(0), accm = T(0);
                for (int m = 0; m < nv; ++m) {
                    accp += e.Lm[k][m] * lc.hp[(i - 2 + s) * nv + m];
                    accm += e.Lm[k][m] * lc.hm[(i - 1 + s) * nv + m];
                }
                gp[s][k] = accp;
                gm[s][k] = accm;
            }
    } else {
        // project F and U of cells i-2..i+3, then split each field with its own speed:
        // g+- = (l_k.F +- alpha_k l_k.U)/2
        T alpha_k[4];
        const int kind3[3] = {0, 1, 2}, kind4[4] = {0, 1, 1, 2};   // eigenvalue of each field
        if (P.split == S_LLF) {
            T a = lc.speed[i - 2];
            for (int s = 1; s < 6; ++s) a = tmax(a, lc.speed[i - 2 + s]);
            for (int k = 0; k < nv; ++k) alpha_k[k] = a;
        } else {
            for (int k = 0; k < nv; ++k) alpha_k[k] = alpha_f[nv == 3 ? kind3[k] : kind4[k]];
        }
        for (int s = 0; s < 6; ++s)
            for (int k = 0; k < nv; ++k) {
                T gF = T(0), gU = T(0);
                for (int m = 0; m < nv; ++m) {
                    gF += e.Lm[k][m] * lc.hp[(i - 2 + s) * nv + m];
                    gU += e.Lm[k][m] * lc.hm[(i - 2 + s) * nv + m];
                }
                if (s <= 4) gp[s][k] = cst<T>(1, 2) * (gF + alpha_k[k] * gU);
                if (s >= 1) gm[s - 1][k] = cst<T>(1, 2) * (gF - alpha_k[k] * gU);
            }
    }
    T ghat[4];
    for (int k = 0; k < nv; ++k) {
        T fp[5] = {gp[0][k], gp[1][k], gp[2][k], gp[3][k], gp[4][k]};
        T fm[5] = {gm[0][k], gm[1][k], gm[2][k], gm[3][k], gm[4][k]};
        ghat[k] = weno5(fp, eps, A, P.weights).fhat + weno5_minus(fm, eps, A, P.weights);
    }
    // back-projection F^ = R g^
    for (int m = 0; m < nv; ++m) {
        T acc = e.R[m][0] * ghat[0];
        for (int k = 1; k < nv; ++k) acc += e.R[m][k] * ghat[k];
        Fhat[m] = acc;
    }
}

// Largest |u_n| + c over the interior (one LF alpha per direction); dir 0 = x, 1 = y.
template <class T>
T cell_speed(const Problem& P, const T* U, int64_t nc, int64_t c, int dir) {
    const int nv = nvar_of(P.system);
    T s[4];
    for (int k = 0; k < nv; ++k) s[k] = U[k * nc + c];
    if (dir == 1) std::swap(s[1], s[2]);
    Prim<T> w = primitives(s, nv, T(P.gamma));
    return tabs(w.un) + sound_speed(w, T(P.gamma));
}

template <class T>
T max_wavespeed(const Problem& P, const T* U, int dir) {
    if (P.system == SYS_ADV1D) return tabs(T(P.adv_speed));
    const int64_t nc = int64_t(P.nx) * P.ny;
    T best = T(0);
    for (int64_t c = 0; c < nc; ++c) best = tmax(best, cell_speed(P, U, nc, c, dir));
    return best;
}

// In double the maximum is exact and independent of the order the cells are visited in, so
// the cells can be spread over the OpenMP threads (the other scalars keep the serial scan:
// a dual number's maximum also picks the derivative of the first maximal cell).
template <>
double max_wavespeed<double>(const Problem& P, const double* U, int dir) {
    if (P.system == SYS_ADV1D) return std::fabs(P.adv_speed);
    const int64_t nc = int64_t(P.nx) * P.ny;
    double best = 0.0;
#pragma omp parallel if (nc > 8192)
    {
        double mine = 0.0;
#pragma omp for schedule(static) nowait
        for (int64_t c = 0; c < nc; ++c) mine = tmax(mine, cell_speed(P, U, nc, c, dir));
#pragma omp critical
        best = tmax(best, mine);
    }
    return best;
}

// Largest |lambda| of each eigenvalue kind (0: u_n - c, 1: u_n, 2: u_n + c) over the
// interior: the per-field LF speeds.
template <class T>
void max_field_speeds(const Problem& P, const T* U, int dir, T* best) {
    const int nv = nvar_of(P.system);
    const int64_t nc = int64_t(P.nx) * P.ny;
    for (int k = 0; k < 3; ++k) best[k] = T(0);
    for (int64_t c = 0; c < nc; ++c) {
        T s[4];
        for (int k = 0; k < nv; ++k) s[k] = U[k * nc + c];
        if (dir == 1) std::swap(s[1], s[2]);
        Prim<T> w = primitives(s, nv, T(P.gamma));
        const T cs = sound_speed(w, T(P.gamma));
        best[0] = tmax(best[0], tabs(w.un - cs));
        best[1] = tmax(best[1], tabs(w.un));
        best[2] = tmax(best[2], tabs(w.un + cs));
    }
}

// The speeds a splitting needs for one stage input: the global LF speeds per direction and,
// for S_LF_FIELD, the per-field ones (x then y, three kinds each).
template <class T> struct Speeds { T ax, ay; T fx[3], fy[3]; };

template <class T>
Speeds<T> stage_speeds(const Problem& P, const T* U) {
    Speeds<T> a{};
    a.ax = max_wavespeed(P, U, 0);
    a.ay = P.system == SYS_EULER2D ? max_wavespeed(P, U, 1) : T(0);
    if (P.split == S_LF_FIELD && P.system != SYS_ADV1D) {
        max_field_speeds(P, U, 0, a.fx);
        if (P.system == SYS_EULER2D) max_field_speeds(P, U, 1, a.fy);
    }
    return a;
}

// Semi-discrete right-hand side, Eq. (2) (and its 2D form, Sec. 4.4):
// Lout = -(F^_{i+1/2} - F^_{i-1/2})/dx [- (G^_{j+1/2} - G^_{j-1/2})/dy].
// `a` holds the LF speeds of this stage input.
template <class T>
void rhs_with_speeds(const Problem& P, const T* U, T* Lout, const Speeds<T>& a) {
    const int nv = nvar_of(P.system);
    const int64_t nx = P.nx, ny = P.ny, nc = nx * ny;
    // x-sweep, one grid row at a time; the rows are spread over the OpenMP threads, or, for a
    // single row (1D), its cells and interfaces are
    auto x_row = [&](int64_t j, bool par) {
        std::vector<T> line((nx + 6) * nv), flux((nx + 1) * nv);
        LineCells<T> lc;
        for (int64_t p = 0; p < nx + 6; ++p) {
            int64_t src = ghost_src(p - 3, nx, P.bc_x);
            for (int k = 0; k < nv; ++k) line[p * nv + k] = U[k * nc + j * nx + src];
            if (nv > 1 && ghost_mirrored(p - 3, nx, P.bc_x)) line[p * nv + 1] = -line[p * nv + 1];
        }
        line_cells(P, line.data(), nx + 6, nv, a.ax, lc, par);
#pragma omp parallel for schedule(static) if (par && nx > 4096)
        for (int64_t f = 0; f <= nx; ++f)   // interface f - 1/2, between padded cells f+2, f+3
            interface_flux(P, lc, nv, f + 2, &flux[f * nv], a.fx);
        for (int64_t i = 0; i < nx; ++i)
            for (int k = 0; k < nv; ++k)
                Lout[k * nc + j * nx + i] = -((flux[(i + 1) * nv + k] - flux[i * nv + k]) / T(P.dx));
    };
    if (ny == 1) {
        x_row(0, true);
    } else {
#pragma omp parallel for schedule(static) if (nc > 4096)
        for (int64_t j = 0; j < ny; ++j) x_row(j, false);
    }
    if (P.system != SYS_EULER2D) return;
    // y-sweep, one grid column at a time, state permuted to (rho, rho v, rho u, E)
#pragma omp parallel for schedule(static) if (nc > 4096)
    for (int64_t i = 0; i < nx; ++i) {
        std::vector<T> line((ny + 6) * nv), flux((ny + 1) * nv);
        LineCells<T> lc;
        const int perm[4] = {0, 2, 1, 3};
        for (int64_t p = 0; p < ny + 6; ++p) {
            int64_t src = ghost_src(p - 3, ny, P.bc_y);
            for (int k = 0; k < nv; ++k) line[p * nv + k] = U[perm[k] * nc + src * nx + i];
            if (ghost_mirrored(p - 3, ny, P.bc_y)) line[p * nv + 1] = -line[p * nv + 1];
        }
        line_cells(P, line.data(), ny + 6, nv, a.ay, lc);
        for (int64_t f = 0; f <= ny; ++f)
            interface_flux(P, lc, nv, f + 2, &flux[f * nv], a.fy);
        for (int64_t j = 0; j < ny; ++j)
            for (int k = 0; k < nv; ++k)
                Lout[perm[k] * nc + j * nx + i] = Lout[perm[k] * nc + j * nx + i]
                                                - (flux[(j + 1) * nv + k] - flux[j * nv + k]) / T(P.dy);
    }
}

template <class T>
void rhs(const Problem& P, const T* U, T* Lout) {
    rhs_with_speeds(P, U, Lout, stage_speeds(P, U));
}

// CFL time step: 1D Sec. 4.3, 2D Sec. 4.4, advection dx*cfl/|a|.
inline double cfl_dt(const Problem& P, const double* U) {
    double ax = max_wavespeed<double>(P, U, 0);
    if (P.system != SYS_EULER2D) return P.cfl * P.dx / ax;
    double ay = max_wavespeed<double>(P, U, 1);
    double tx = P.dx / ax, ty = P.dy / ay;
    return P.cfl * tx * ty / (tx + ty);
}

// Third-order TVD (SSP) Runge-Kutta of Shu and Osher (cited in Sec. 4):
//   U1 = Un + dt L(Un);  U2 = 3/4 Un + 1/4 (U1 + dt L(U1));  Un+1 = 1/3 Un + 2/3 (U2 + dt L(U2)).
// `L` is any callable (const double* in, double* out).
template <class RhsFn>
void ssp_rk3(int64_t n, double* U, double dt, RhsFn L) {
    std::vector<double> U0(U, U + n), U1(n), U2(n), K(n);
    L(U0.data(), K.data());
#pragma omp parallel for schedule(static) if (n > 65536)
    for (int64_t c = 0; c < n; ++c) U1[c] = U0[c] + dt * K[c];
    L(U1.data(), K.data());
#pragma omp parallel for schedule(static) if (n > 65536)
    for (int64_t c = 0; c < n; ++c) U2[c] = 0.75 * U0[c] + 0.25 * (U1[c] + dt * K[c]);
    L(U2.data(), K.data());
#pragma omp parallel for schedule(static) if (n > 65536)
    for (int64_t c = 0; c < n; ++c) U[c] = U0[c] / 3.0 + 2.0 / 3.0 * (U2[c] + dt * K[c]);
}

// The same SSP-RK3 on any scalar type with a fixed step (used by the JVP instantiation).
template <class T>
void ssp_rk3_fixed(const Problem& P, std::vector<T>& U, double dt_d) {
    const size_t n = U.size();
    const T dt{dt_d};
    std::vector<T> U0(U), U1(n), U2(n), K(n);
    rhs<T>(P, U0.data(), K.data());
    for (size_t c = 0; c < n; ++c) U1[c] = U0[c] + dt * K[c];
    rhs<T>(P, U1.data(), K.data());
    for (size_t c = 0; c < n; ++c) U2[c] = T(0.75) * U0[c] + T(0.25) * (U1[c] + dt * K[c]);
    rhs<T>(P, U2.data(), K.data());
    for (size_t c = 0; c < n; ++c) U[c] = U0[c] / T(3.0) + T(2.0) / T(3.0) * (U2[c] + dt * K[c]);
}

}  // namespace orc

using namespace orc;

// Sec. 4.1 critical-point test: error of (f^+_{1/2} - f^+_{-1/2})/dx against f'(0) for
// f(x) = x^k e^x sampled at x_j = j dx, reconstructed directly (no flux splitting).
template <class T>
static T exp_series(T x) {
    T sum = T(1), term = T(1);
    for (int n = 1; n < 60; ++n) {
        term = term * x / T(n);
        sum = sum + term;
    }
    return sum;
}

template <class T>
static double critical_point_error(int k, double dx_d, int kind, double eps_d) {
    const T dx = T(dx_d), eps = T(eps_d), A = T(10);
    T f[7];   // f_{-3} .. f_{3}
    for (int j = -3; j <= 3; ++j) {
        T x = T(j) * dx, xk = T(1);
        for (int m = 0; m < k; ++m) xk = xk * x;
        f[j + 3] = xk * exp_series(x);
    }
    T fr = weno5(&f[1], eps, A, kind).fhat;   // f^+_{1/2} from f_{-2..2}
    T fl = weno5(&f[0], eps, A, kind).fhat;   // f^+_{-1/2} from f_{-3..1}
    T d = (fr - fl) / dx;
    T exact = k == 1 ? T(1) : T(0);
    return double(tabs(d - exact));
}


// =======================================================================================
// C entry points (ctypes)
// =======================================================================================
extern "C" {

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

// All intermediates of one reconstruction f^+_{i+1/2} from f[0..4] = f_{i-2..i+2}.
// out: q0 q1 q2 IS0 IS1 IS2 tau5 tau8 C alpha0 alpha1 alpha2 omega0 omega1 omega2 fhat
void oracle_weno5_parts(const double* f, double eps, double A, int kind, double* out) {
    WenoParts<double> r = weno5(f, eps, A, kind);
    double v[16] = {r.q[0], r.q[1], r.q[2], r.IS[0], r.IS[1], r.IS[2], r.tau5, r.tau8, r.C,
                    r.alpha[0], r.alpha[1], r.alpha[2], r.omega[0], r.omega[1], r.omega[2], r.fhat};
    std::memcpy(out, v, sizeof v);
}

// Reconstruction over a padded line: f_padded[n+6] (three ghosts each side, already filled),
// fhat[n+1] at the interfaces x_{j-1/2}, j = 0..n.  side = +1: f^+, side = -1: f^- (mirror).
void oracle_reconstruct(const double* f_padded, int64_t n, double* fhat, int side,
                        double eps, double A, int kind) {
    for (int64_t j = 0; j <= n; ++j) {
        // interface j - 1/2 lies between padded cells j+2 and j+3 (i = padded j+2)
        if (side > 0) fhat[j] = weno5(&f_padded[j], eps, A, kind).fhat;
        else fhat[j] = weno5_minus(&f_padded[j + 1], eps, A, kind);
    }
}

// The same reconstruction evaluated in binary128 (inputs and eps converted exactly, results
// rounded to double): its exponent range (about 1e+-4932) holds every intermediate of Eq.
// (function) and Eq. (new) for any double input, so it is the reference where the plain
// double evaluation overflows (e.g. C when tau5 = 0 and the indicators exceed about 1e114).
void oracle_reconstruct_quad(const double* f_padded, int64_t n, double* fhat, int side, double eps,
                             double A, int kind) {
    std::vector<Quad> f(n + 6);
    for (int64_t j = 0; j < n + 6; ++j) f[j] = Quad(f_padded[j]);
    for (int64_t j = 0; j <= n; ++j) {
        const Quad r = side > 0 ? weno5(&f[j], Quad(eps), Quad(A), kind).fhat
                                : weno5_minus(&f[j + 1], Quad(eps), Quad(A), kind);
        fhat[j] = double(r);
    }
}

double oracle_critical_point_error(int k, double dx, int kind, double eps, int quad) {
    return quad ? critical_point_error<Quad>(k, dx, kind, eps)
                : critical_point_error<double>(k, dx, kind, eps);
}

// Ghost fill of one padded line (n interior values at f_padded[3..n+2]).
void oracle_fill_ghosts_line(double* f_padded, int64_t n, int bc) {
    for (int g = 1; g <= 3; ++g) {
        f_padded[3 - g] = f_padded[3 + ghost_src(-g, n, bc)];
        f_padded[n + 2 + g] = f_padded[3 + ghost_src(n - 1 + g, n, bc)];
    }
}

double oracle_max_wavespeed(const Problem* P, const double* U, int dir) {
    return max_wavespeed<double>(*P, U, dir);
}

double oracle_cfl_dt(const Problem* P, const double* U) { return cfl_dt(*P, U); }

void oracle_rhs(const Problem* P, const double* U, double* Lout) { rhs<double>(*P, U, Lout); }

// One SSP-RK3 step in place.  dt > 0: fixed step; dt <= 0: CFL step from Un.
// t_remaining > 0 clips the step.  Returns the step taken.
double oracle_rk3_step(const Problem* P, double* U, double dt, double t_remaining) {
    if (!(dt > 0)) dt = cfl_dt(*P, U);
    if (t_remaining > 0 && dt > t_remaining) dt = t_remaining;
    const int64_t n = int64_t(nvar_of(P->system)) * P->nx * P->ny;
    ssp_rk3(n, U, dt, [&](const double* Uin, double* K) { rhs<double>(*P, Uin, K); });
    return dt;
}

// Advance to time T.  dt > 0: ceil(T/dt) fixed steps, the last one landing on T;
// dt <= 0: CFL steps clipped at T.  Returns the number of steps.
int64_t oracle_run(const Problem* P, double* U, double T, double dt) {
    if (dt > 0) {
        const int64_t n = int64_t(std::ceil(T / dt - 1e-9));
        for (int64_t k = 0; k < n; ++k)
            oracle_rk3_step(P, U, k == n - 1 ? T - double(k) * dt : dt, 0.0);
        return n;
    }
    double t = 0;
    int64_t steps = 0;
    while (t < T * (1 - 1e-14)) {
        t += oracle_rk3_step(P, U, 0.0, T - t);
        ++steps;
    }
    return steps;
}

// The RK3 combination alone on the scalar ODE u' = lambda u (stability-polynomial pin).
double oracle_rk3_linear(double lambda, double dt, double u0) {
    double u = u0;
    ssp_rk3(1, &u, dt, [&](const double* in, double* out) { out[0] = lambda * in[0]; });
    return u;
}

// Roe state and eigenvectors between two states (nv = 3 or 4, direction frame).
// out: un ut H c, then R (4x4 row-major), then Lm (4x4 row-major): 36 values.
void oracle_roe_eigen(const double* UL, const double* UR, int nv, double gamma, double* out) {
    Eigen<double> e = roe_eigen<double>(UL, UR, nv, gamma);
    out[0] = e.un; out[1] = e.ut; out[2] = e.H; out[3] = e.c;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            out[4 + i * 4 + j] = e.R[i][j];
            out[20 + i * 4 + j] = e.Lm[i][j];
        }
}

void oracle_normal_flux(const double* U, int nv, double gamma, double* F) {
    Prim<double> w = primitives<double>(U, nv, gamma);
    normal_flux<double>(U, w, nv, F);
}

// Algorithmic floating-point operations of one RHS evaluation on an nx x ny periodic
// grid (alpha reduction included), counted by running the oracle on OpCount scalars.
// out: add mul div sqrt cmp (totals).
void oracle_opcount_rhs_variant(int system, int nx, int ny, int weights, int split, double* out) {
    Problem P{};
    P.system = system; P.nx = nx; P.ny = ny; P.bc_x = BC_PERIODIC; P.bc_y = BC_PERIODIC;
    P.weights = weights; P.split = split; P.dx = 0.1; P.dy = 0.1; P.gamma = 1.4; P.eps = 1e-40; P.A = 10;
    P.cfl = 0.5; P.adv_speed = 1.0;
    const int nv = nvar_of(system);
    const int64_t nc = int64_t(nx) * ny;
    std::vector<OpCount> U(nv * nc), L(nv * nc);
    for (int64_t c = 0; c < nc; ++c) {
        double x = 0.37 * double(c % nx) + 0.11 * double(c / nx);
        U[c] = OpCount(1.0 + 0.2 * std::sin(x));
        if (nv >= 3) {
            U[nc + c] = OpCount(0.3 * std::cos(x));
            if (nv == 4) U[2 * nc + c] = OpCount(-0.2 * std::sin(2 * x));
            U[(nv - 1) * nc + c] = OpCount(2.5 + 0.1 * std::cos(3 * x));
        }
    }
    g_tally = OpTally();
#ifdef _OPENMP
    int saved = omp_get_max_threads();
    omp_set_num_threads(1);
#endif
    rhs<OpCount>(P, U.data(), L.data());
#ifdef _OPENMP
    omp_set_num_threads(saved);
#endif
    out[0] = double(g_tally.add); out[1] = double(g_tally.mul); out[2] = double(g_tally.div);
    out[3] = double(g_tally.sqrt_); out[4] = double(g_tally.cmp);
}

void oracle_opcount_rhs(int system, int nx, int ny, double* out) {
    oracle_opcount_rhs_variant(system, nx, ny, W_ZN, S_LF, out);
}

// Algorithmic operations of the pieces of one RHS, counted on OpCount scalars (add+mul+div
// +sqrt; comparisons apart): out[0] one interface flux, out[1] the per-cell split-flux
// and Roe ingredients of one sweep (per cell), out[2] one cell's LF-speed evaluation
// (both directions in 2D), out[3] one cell's flux difference per direction,
// out[4..8] the comparison counts of the same pieces.
void oracle_opcount_parts_variant(int system, int weights, int split, double* out) {
    Problem P{};
    P.system = system; P.nx = 8; P.ny = 1; P.bc_x = BC_PERIODIC; P.bc_y = BC_PERIODIC;
    P.weights = weights; P.split = split; P.dx = 0.1; P.dy = 0.1; P.gamma = 1.4; P.eps = 1e-40; P.A = 10;
    P.cfl = 0.5; P.adv_speed = 1.0;
    const int nv = nvar_of(system);
    std::vector<OpCount> line(14 * nv);
    for (int c = 0; c < 14; ++c) {
        double x = 0.37 * c;
        line[c * nv] = OpCount(1.0 + 0.2 * std::sin(x));
        if (nv >= 3) {
            line[c * nv + 1] = OpCount(0.3 * std::cos(x));
            if (nv == 4) line[c * nv + 2] = OpCount(-0.2 * std::sin(2 * x));
            line[c * nv + nv - 1] = OpCount(2.5 + 0.1 * std::cos(3 * x));
        }
    }
    auto total = [](const OpTally& t) { return double(t.add + t.mul + t.div + t.sqrt_); };
    LineCells<OpCount> lc;
    g_tally = OpTally();
    line_cells(P, line.data(), 14, nv, OpCount(2.0), lc);
    out[1] = total(g_tally) / 14.0; out[5] = double(g_tally.cmp) / 14.0;
    OpCount F[4];
    OpCount af[3] = {OpCount(1.0), OpCount(1.5), OpCount(2.0)};
    g_tally = OpTally();
    interface_flux(P, lc, nv, 5, F, af);
    out[0] = total(g_tally); out[4] = double(g_tally.cmp);
    std::vector<OpCount> U(nv * 8);
    for (int k = 0; k < nv; ++k)
        for (int c = 0; c < 8; ++c) U[k * 8 + c] = line[c * nv + k];
    g_tally = OpTally();
    if (system != SYS_ADV1D) {
        P.nx = 8;
        max_wavespeed<OpCount>(P, U.data(), 0);
        if (system == SYS_EULER2D) max_wavespeed<OpCount>(P, U.data(), 1);
        if (split == S_LF_FIELD) {
            OpCount fs[3];
            max_field_speeds<OpCount>(P, U.data(), 0, fs);
            if (system == SYS_EULER2D) max_field_speeds<OpCount>(P, U.data(), 1, fs);
        }
    }
    out[2] = total(g_tally) / 8.0; out[6] = double(g_tally.cmp) / 8.0;
    // flux difference: -(F_{i+1/2} - F_{i-1/2}) / dx per variable
    g_tally = OpTally();
    OpCount d = -((F[0] - F[0]) / OpCount(0.1));
    (void)d;
    out[3] = total(g_tally) * nv; out[7] = 0.0; out[8] = 0.0;
}

// Steger-Warming split flux F+ (sign > 0) or F- (sign < 0) of one state (direction frame).
void oracle_steger_warming(const double* U, int nv, double gamma, int sign, double* F) {
    Prim<double> w = primitives<double>(U, nv, gamma);
    steger_warming<double>(w, nv, gamma, sign > 0 ? 1 : -1, F);
}

// Largest |lambda| of eigenvalue kind (0: u_n - c, 1: u_n, 2: u_n + c) over the grid.
double oracle_field_speed(const Problem* P, const double* U, int dir, int kind) {
    double best[3];
    max_field_speeds<double>(*P, U, dir, best);
    return best[kind];
}

// RHS with the LF speeds given: sp = (alpha_x, alpha_y, fx0, fx1, fx2, fy0, fy1, fy2).
void oracle_rhs_speeds(const Problem* P, const double* U, const double* sp, double* Lout) {
    Speeds<double> a{};
    a.ax = sp[0]; a.ay = sp[1];
    for (int k = 0; k < 3; ++k) { a.fx[k] = sp[2 + k]; a.fy[k] = sp[5 + k]; }
    rhs_with_speeds<double>(*P, U, Lout, a);
}

void oracle_opcount_parts(int system, double* out) { oracle_opcount_parts_variant(system, W_ZN, S_LF, out); }

// Jacobian-vector products of the discrete scheme (forward mode, Dual scalars).
// rhs: L = rhs(U), dL = J(U) dU (the LF speed differentiated through its argmax cell).
void oracle_rhs_jvp(const Problem* P, const double* U, const double* dU, double* L, double* dL) {
    const int64_t n = int64_t(nvar_of(P->system)) * P->nx * P->ny;
    std::vector<Dual> u(n), l(n);
    for (int64_t c = 0; c < n; ++c) u[c] = Dual(U[c], dU[c]);
    rhs<Dual>(*P, u.data(), l.data());
    for (int64_t c = 0; c < n; ++c) { L[c] = l[c].v; dL[c] = l[c].d; }
}

// The same product evaluated in binary128 (reference derivative where the double one is
// ill-conditioned, e.g. at IS_0 ~ IS_2 where the derivative of C divides by (tau5 + eps)^2).
void oracle_rhs_jvp_quad(const Problem* P, const double* U, const double* dU, double* L, double* dL) {
    const int64_t n = int64_t(nvar_of(P->system)) * P->nx * P->ny;
    std::vector<DualQ> u(n), l(n);
    for (int64_t c = 0; c < n; ++c) u[c] = DualQ(Quad(U[c]), Quad(dU[c]));
    rhs<DualQ>(*P, u.data(), l.data());
    for (int64_t c = 0; c < n; ++c) { L[c] = double(l[c].v); dL[c] = double(l[c].d); }
}

// `steps` SSP-RK3 steps with the fixed step dt, in place for U and the tangent dU.
void oracle_rollout_jvp(const Problem* P, double* U, double* dU, double dt, int64_t steps) {
    const int64_t n = int64_t(nvar_of(P->system)) * P->nx * P->ny;
    std::vector<Dual> u(n);
    for (int64_t c = 0; c < n; ++c) u[c] = Dual(U[c], dU[c]);
    for (int64_t k = 0; k < steps; ++k) ssp_rk3_fixed<Dual>(*P, u, dt);
    for (int64_t c = 0; c < n; ++c) { U[c] = u[c].v; dU[c] = u[c].d; }
}

// The same rollout derivative in binary128.
void oracle_rollout_jvp_quad(const Problem* P, double* U, double* dU, double dt, int64_t steps) {
    const int64_t n = int64_t(nvar_of(P->system)) * P->nx * P->ny;
    std::vector<DualQ> u(n);
    for (int64_t c = 0; c < n; ++c) u[c] = DualQ(Quad(U[c]), Quad(dU[c]));
    for (int64_t k = 0; k < steps; ++k) ssp_rk3_fixed<DualQ>(*P, u, dt);
    for (int64_t c = 0; c < n; ++c) { U[c] = double(u[c].v); dU[c] = double(u[c].d); }
}

}  // extern "C"
