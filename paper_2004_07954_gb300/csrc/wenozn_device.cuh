// Device-side building blocks of the WENO-ZN solver (FP64, sm_103a).
//
// The arithmetic here is the paper's, rearranged for a GPU whose FP64 pipe is the scarce
// resource: constants are folded, the three un-normalised weights are brought to a common
// denominator so that one division per reconstruction remains, and comparisons of
// non-negative indicators run on the integer pipe.  Every rearrangement is exact algebra;
// only the rounding differs from the plain evaluation order.
#pragma once

#include <cmath>
#include <cstdint>

namespace wz {

// ------------------------------------------------------------------------------------
// Fifth-order WENO-ZN reconstruction f^+_{i+1/2} from (a, b, c, d, e) = f_{i-2 .. i+2}.
//
//   Eq. (4)        q_0 = (2a - 7b + 11c)/6, q_1 = (-b + 5c + 2d)/6, q_2 = (2c + 5d - e)/6
//   Eq. (isjiang)  IS_k = 13/12 s_k^2 + 1/4 t_k^2 with s_k the second difference and t_k
//                  the one-sided first difference of sub-stencil k
//   Eq. (tau)      tau5 = |IS_0 - IS_2|
//   Eq. (tau8)     tau8 = (a - 4b + 6c - 4d + e)^2
//   Eq. (function) C = A ((IS_0 + IS_2 - tau5 + eps)/(tau5 + eps))^2
//   Eq. (new)      alpha_k = c_k (C + tau8/(IS_k + eps)),  c = (1, 6, 3)/10
//   Eq. (3)        f^ = sum_k alpha_k q_k / sum_k alpha_k
//
// Evaluation (exact algebra; only the rounding differs from the plain order):
//  * with the first differences D1 = a - b, D2 = b - c, D3 = c - d, D4 = d - e, the second
//    differences s_0 = D1 - D2, s_1 = D2 - D3, s_2 = D3 - D4 and the one-sided ones
//    t_0 = D1 - 3 D2 = a - 4b + 3c, t_1 = D2 + D3 = b - d, t_2 = 3 D3 - D4 = 3c - 4d + e (equal
//    inputs give exact zeros, so constant data keep exactly the linear weights), the
//    sub-stencil fluxes are
//    q_k = c + s_k/12 + t_k/4 (k = 0) and c + s_k/12 - t_k/4 (k = 1, 2), and since the
//    normalised weights sum to one the centre value is taken out: f^ = c + sum w_k (q_k - c);
//  * indicators are carried scaled by 4 together with eps: b_k = 4 (IS_k + eps)
//    = 13/3 s_k^2 + t_k^2 + 4 eps, so C and tau8/(IS_k + eps) = 4 tau8 / b_k are unchanged;
//  * IS_0 + IS_2 - tau5 = 2 min(IS_0, IS_2), i.e. 4 (IS_0 + IS_2 - tau5 + eps) = 2 min(b) - 4 eps
//    = m and 4 (tau5 + eps) = max(b) - min(b) + 4 eps = P; min/max of the non-negative b
//    run on the integer pipe;
//  * every alpha_k is multiplied by P^2 b_0 b_1 b_2 / (A c_k) and the common factor divided
//    out: a_k = m^2 b_0 b_1 b_2 + (kappa d4 P)^2 prod_{j != k} b_j with d4 the fourth
//    difference and kappa = 2 / sqrt(A) (A > 0), all positive (a_k >= (4 eps)^5 > 0); the
//    optimal weights (1, 6, 3)/10
//    then enter through 6 q_1 and 3 q_2 and the denominator a_0 + 6 a_1 + 3 a_2, leaving one
//    division per reconstruction.  The fourth difference is d4 = t0 + t2.
//
// Range.  The a_k are fifth powers of the indicators, so for stencils whose differences
// exceed about 2^88 they overflow, and for data far below the scale of eps (differences
// under about sqrt(eps) times 1e-100) the numerator underflows.  Every quantity above is
// homogeneous once eps is scaled with the data: with the first differences multiplied by s
// and eps by s^2, each b_k scales by s^2, each a_k by s^10 and num/den by s.  So the fast
// evaluation is kept, its num and den are checked on the integer pipe, and in the rare case
// they left the double range the weights are evaluated again on the differences scaled by
// an exact power of two that brings the largest indicator near 2^100 (zn_correction_rescaled;
// the Jiang-Shu variant divides the smallest indicator out instead).
// With 1e-60 <= eps <= 1 and 1e-6 <= A <= 1e6 the result is then finite and accurate for
// every stencil whose first differences stay below 2^440 (about 2.8e132) in magnitude.
// ------------------------------------------------------------------------------------
// Reciprocal of a positive, normal double: start from the hardware approximation
// r0 (rcp.approx.ftz.f64, about 23 correct bits), form e = 1 - d r0 and take one step of
// the cubically convergent series 1/d = r0 (1 + e + e^2 + ...) truncated after e^2
// (Householder's third-order iteration): the relative error becomes about e^3 ~ 2^-69, so
// the result is within about one ulp of 1/d.  Used where d is known to be positive and normal.
__host__ __device__ __forceinline__ double rcp_nr(double d) {
#ifdef __CUDA_ARCH__
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    const double e = fma(-d, r, 1.0);
    return fma(r, fma(e, e, e), r);
#else
    return 1.0 / d;
#endif
}

// WENO-ZN numerator and denominator of f^ - c from the first differences D1..D4 (the
// evaluation described above).
__host__ __device__ __forceinline__ void zn_num_den_tb(double D1, double D2, double D3, double D4, double t0,
                                                       double t2, double b0, double b1, double b2, double eps4,
                                                       double kappa, double& num, double& den);

__host__ __device__ __forceinline__ void zn_num_den(double D1, double D2, double D3, double D4, double eps4,
                                                    double kappa, double& num, double& den) {
    // second (s_k) and one-sided (t_k) differences from the first: equal inputs give exact zeros
    const double s0 = D1 - D2, s1 = D2 - D3, s2 = D3 - D4;
    const double t0 = fma(-3.0, D2, D1), t1 = D2 + D3, t2 = fma(3.0, D3, -D4);
    const double k13_3 = 13.0 / 3.0;
    const double b0 = fma(k13_3 * s0, s0, fma(t0, t0, eps4));   // 4 (IS_0 + eps)
    const double b1 = fma(k13_3 * s1, s1, fma(t1, t1, eps4));
    const double b2 = fma(k13_3 * s2, s2, fma(t2, t2, eps4));
    zn_num_den_tb(D1, D2, D3, D4, t0, t2, b0, b1, b2, eps4, kappa, num, den);
}

// The same from the scaled indicators b_k = 4 (IS_k + eps) and the one-sided differences
// t_0, t_2 (callers that share parts of the indicators between neighbouring stencils).
__host__ __device__ __forceinline__ void zn_num_den_tb(double D1, double D2, double D3, double D4, double t0,
                                                       double t2, double b0, double b1, double b2, double eps4,
                                                       double kappa, double& num, double& den) {
    const double d4 = t0 + t2;                                  // a - 4b + 6c - 4d + e
    // non-negative doubles order like their bit patterns: min/max on the integer pipe
#ifdef __CUDA_ARCH__
    const long long i0 = __double_as_longlong(b0), i2 = __double_as_longlong(b2);
    const double mn = __longlong_as_double(i0 < i2 ? i0 : i2);
    const double mx = __longlong_as_double(i0 < i2 ? i2 : i0);
#else
    const double mn = b0 < b2 ? b0 : b2, mx = b0 < b2 ? b2 : b0;
#endif
    const double P = fma(kappa, mx - mn, kappa * eps4);          // kappa 4 (tau5 + eps)
    const double m = fma(2.0, mn, -eps4);                       // 4 (IS_0 + IS_2 - tau5 + eps)
    const double b01 = b0 * b1, b12 = b1 * b2, b02 = b0 * b2;
    const double X = (m * m) * (b01 * b2);
    const double z = d4 * P;
    const double Y = z * z;
    const double a0 = fma(Y, b12, X);
    const double a1 = fma(Y, b02, X);
    const double a2 = fma(Y, b01, X);
    // q_k - c scaled by the optimal-weight ratios (1, 6, 3); the weights sum to one, so
    // f^ = c + sum a_k (q_k - c) / sum a_k
    // from the first differences: q_0 - c = D1/3 - 5 D2/6, 6 (q_1 - c) = -(D2 + 2 D3),
    // 3 (q_2 - c) = D4/2 - 2 D3
    const double q0 = fma(1.0 / 3.0, D1, (-5.0 / 6.0) * D2);
    const double q1n = fma(2.0, D3, D2);
    const double q2 = fma(-2.0, D3, 0.5 * D4);
    num = fma(a0, q0, fma(-a1, q1n, a2 * q2));
    den = fma(6.0, a1, fma(3.0, a2, a0));
}

// ------------------------------------------------------------------------------------
// The same reconstruction with the weight function chosen at run time (weights: 0 WENO-ZN,
// Eq. (new); 1 WENO-Z with q = 1, Eq. (15); 2 linear (the optimal weights c_k); 3 Jiang-Shu,
// c_k / (IS_k + eps)^2, Sec. 2.1).  All four share the scaled indicators b_k = 4 (IS_k + eps)
// and the common-denominator form f^ = sum a_k q'_k / (a_0 + 6 a_1 + 3 a_2):
//   WENO-Z:  alpha_k / c_k = 1 + tau5/(IS_k + eps) = (b_k + T)/b_k with T = |b_0 - b_2| = 4 tau5;
//            times b_0 b_1 b_2: a_k = b_0 b_1 b_2 + T prod_{j != k} b_j;
//   JS:      alpha_k / c_k = 16 / b_k^2; times (b_0 b_1 b_2)^2 / 16: a_k = (prod_{j != k} b_j)^2;
//   linear:  a_k = 1.
// Each is homogeneous in the data with eps scaled alike, so the range guard above applies.
// ------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ void zn_num_den_w(double D1, double D2, double D3, double D4, double eps4,
                                                      double kappa, int weights, double& num, double& den) {
    if (weights == 0) {
        zn_num_den(D1, D2, D3, D4, eps4, kappa, num, den);
        return;
    }
    const double s0 = D1 - D2, s1 = D2 - D3, s2 = D3 - D4;
    const double t0 = fma(-3.0, D2, D1), t1 = D2 + D3, t2 = fma(3.0, D3, -D4);
    const double k13_3 = 13.0 / 3.0;
    const double k1_12 = 1.0 / 12.0;
    const double q0 = fma(k1_12, s0, 0.25 * t0);
    const double q1 = fma(0.5, s1, -1.5 * t1);
    const double q2 = fma(0.25, s2, -0.75 * t2);
    double a0 = 1.0, a1 = 1.0, a2 = 1.0;
    if (weights != 2) {
        const double b0 = fma(k13_3 * s0, s0, fma(t0, t0, eps4));
        const double b1 = fma(k13_3 * s1, s1, fma(t1, t1, eps4));
        const double b2 = fma(k13_3 * s2, s2, fma(t2, t2, eps4));
        const double b12 = b1 * b2, b02 = b0 * b2, b01 = b0 * b1;
        if (weights == 1) {
            const double T = fabs(b0 - b2);
            const double b012 = b01 * b2;
            a0 = fma(T, b12, b012);
            a1 = fma(T, b02, b012);
            a2 = fma(T, b01, b012);
        } else {
            a0 = b12 * b12;
            a1 = b02 * b02;
            a2 = b01 * b01;
        }
    }
    num = fma(a0, q0, fma(a1, q1, a2 * q2));
    den = fma(6.0, a1, fma(3.0, a2, a0));
}

// Whether the fast evaluation left the double range: den (a sum of positive terms) not a
// positive normal number, num not finite, or num flushed to zero or subnormal by underflow
// while the data are not constant.  Integer operations on the bit patterns only.
__host__ __device__ __forceinline__ bool zn_out_of_range(double num, double den, double D1, double D2, double D3,
                                                         double D4) {
#ifdef __CUDA_ARCH__
    const unsigned ed = (unsigned(__double2hiint(den)) >> 20) & 0x7ffu;
    const unsigned en = (unsigned(__double2hiint(num)) >> 20) & 0x7ffu;
    if (ed - 1u < 0x7feu && en != 0x7ffu && en != 0u) return false;
    const unsigned long long any = (__double_as_longlong(D1) | __double_as_longlong(D2) |
                                    __double_as_longlong(D3) | __double_as_longlong(D4)) << 1;   // sign dropped
    return !(ed - 1u < 0x7feu && en != 0x7ffu) || any != 0ull;
#else
    if (!(den > 0.0) || !std::isnormal(den) || !std::isfinite(num)) return true;
    return (num == 0.0 || !std::isnormal(num)) && (D1 != 0.0 || D2 != 0.0 || D3 != 0.0 || D4 != 0.0);
#endif
}

// f^ - c re-evaluated where the fast evaluation left the double range; exact algebra.
//  * WENO-ZN, WENO-Z: the differences scaled by 2^k and eps by 2^2k, with k chosen so that the
//    largest scaled indicator lies in [2^99, 2^102); the scaling is undone on the quotient.
//    Every a_k keeps at most one factor near eps against the largest indicators (sub-stencils
//    0 and 2 share f_i, so they cannot both be flat unless all three are), so nothing of
//    weight underflows.
//  * Jiang-Shu: a_k = (prod_{j != k} b_j)^2 spans the square of the indicators' ratio, which
//    no common scale keeps in range; with the smallest indicator divided out instead,
//    a_k = (b_min / b_k)^2 lies in (0, 1].
__host__ __device__ __forceinline__ double zn_correction_rescaled(double D1, double D2, double D3, double D4,
                                                                  double eps4, double kappa, int weights) {
    const double s0 = D1 - D2, s1 = D2 - D3, s2 = D3 - D4;
    const double t0 = fma(-3.0, D2, D1), t1 = D2 + D3, t2 = fma(3.0, D3, -D4);
    const double k13_3 = 13.0 / 3.0;
    const double b0 = fma(k13_3 * s0, s0, fma(t0, t0, eps4));
    const double b1 = fma(k13_3 * s1, s1, fma(t1, t1, eps4));
    const double b2 = fma(k13_3 * s2, s2, fma(t2, t2, eps4));
    if (weights == 3) {
        const double bm = fmin(b0, fmin(b1, b2));
        const double r0 = bm * rcp_nr(b0), r1 = bm * rcp_nr(b1), r2 = bm * rcp_nr(b2);
        const double a0 = r0 * r0, a1 = r1 * r1, a2 = r2 * r2;
        const double q0 = fma(1.0 / 12.0, s0, 0.25 * t0);
        const double q1 = fma(0.5, s1, -1.5 * t1);
        const double q2 = fma(0.25, s2, -0.75 * t2);
        const double num = fma(a0, q0, fma(a1, q1, a2 * q2));
        const double den = fma(6.0, a1, fma(3.0, a2, a0));
        return num * rcp_nr(den);
    }
    // the largest indicator 4 (IS_k + eps) of the unscaled data fixes the scale
    const double B = fmax(b0, fmax(b1, b2));
    int eb = 0;
    (void)frexp(B, &eb);                       // B in [2^(eb-1), 2^eb)
    int k = (101 - eb) >> 1;                   // B 2^2k in [2^99, 2^102)
    k = k < -500 ? -500 : (k > 500 ? 500 : k);
    const double s = ldexp(1.0, k), si = ldexp(1.0, -k);
    double num, den;
    zn_num_den_w(D1 * s, D2 * s, D3 * s, D4 * s, (eps4 * s) * s, kappa, weights, num, den);
    return (num * rcp_nr(den)) * si;
}

// f^ = c + num / den, with the rescaled evaluation when the fast one left the double range.
// den is then a positive normal number (eps >= 1e-60 makes den >= 10 (4 eps)^5), so the
// Newton reciprocal applies.
// base + (f^ - c) from the stencil's first differences D1..D4 (f^ - c depends on nothing
// else), so that a caller holding the differences and several centre values adds them once.
__host__ __device__ __forceinline__ double zn_flux_d(double D1, double D2, double D3, double D4, double base,
                                                     double eps4, double kappa) {
    double num, den;
    zn_num_den(D1, D2, D3, D4, eps4, kappa, num, den);
    if (zn_out_of_range(num, den, D1, D2, D3, D4))
        return base + zn_correction_rescaled(D1, D2, D3, D4, eps4, kappa, 0);
    return fma(num, rcp_nr(den), base);
}

// zn_flux_d with the second-difference part of the indicators given, S_k = (13/3) s_k^2 + 4 eps
// (s_k the second difference of sub-stencil k): b_k = t_k^2 + S_k.  NEG: base - (f^ - c) of
// the differences D1..D4, which is base + (f^ - c) of the negated differences (f^ - c is odd
// in them: the numerator changes sign, the denominator and the range guard do not).
template <bool NEG = false>
__host__ __device__ __forceinline__ double zn_flux_ds(double D1, double D2, double D3, double D4, double S0,
                                                      double S1, double S2, double base, double eps4,
                                                      double kappa) {
    const double t0 = fma(-3.0, D2, D1), t1 = D2 + D3, t2 = fma(3.0, D3, -D4);
    double num, den;
    zn_num_den_tb(D1, D2, D3, D4, t0, t2, fma(t0, t0, S0), fma(t1, t1, S1), fma(t2, t2, S2), eps4, kappa, num,
                  den);
    if (zn_out_of_range(num, den, D1, D2, D3, D4)) {
        const double corr = zn_correction_rescaled(D1, D2, D3, D4, eps4, kappa, 0);
        return NEG ? base - corr : base + corr;
    }
    return fma(NEG ? -num : num, rcp_nr(den), base);
}

__host__ __device__ __forceinline__ double zn_flux(double a, double b, double c, double d, double e,
                                                   double eps4, double kappa) {
    return zn_flux_d(a - b, b - c, c - d, d - e, c, eps4, kappa);
}

// f^+ + f^- at one interface: plus side from (p0..p4) = h+_{i-2..i+2}, minus side from the
// mirrored stencil (m4, m3, m2, m1, m0) where (m0..m4) = h-_{i-1..i+3} (Sec. 2, the
// "symmetric rule about x_{i+1/2}").
__device__ __forceinline__ double zn_split_flux(double p0, double p1, double p2, double p3, double p4,
                                                double m0, double m1, double m2, double m3, double m4,
                                                double eps4, double kappa) {
    return zn_flux(p0, p1, p2, p3, p4, eps4, kappa) + zn_flux(m4, m3, m2, m1, m0, eps4, kappa);
}

// zn_flux_d with the weight function chosen at run time
__host__ __device__ __forceinline__ double zn_flux_w_d(double D1, double D2, double D3, double D4, double base,
                                                       double eps4, double kappa, int weights) {
    double num, den;
    zn_num_den_w(D1, D2, D3, D4, eps4, kappa, weights, num, den);
    if (zn_out_of_range(num, den, D1, D2, D3, D4))
        return base + zn_correction_rescaled(D1, D2, D3, D4, eps4, kappa, weights);
    return fma(num, rcp_nr(den), base);
}

__host__ __device__ __forceinline__ double zn_flux_w(double a, double b, double c, double d, double e,
                                                     double eps4, double kappa, int weights) {
    return zn_flux_w_d(a - b, b - c, c - d, d - e, c, eps4, kappa, weights);
}

// ------------------------------------------------------------------------------------
// Workspace control block (first 256 bytes of the caller's workspace).
// ------------------------------------------------------------------------------------
struct Ctrl {
    unsigned long long alpha[3][2];       // LF speeds per RK stage slot, as IEEE bit patterns
    unsigned long long alpha_f[3][2][3];  // per-field speeds (slot, direction, |u-c|, |u|, |u+c|)
    double dt;                            // the step the current RK3 step uses
    int32_t status;                       // OR of (1 << wenozn_status) device-detected bits
    int32_t pad0;
    double reserved[6];
};
static_assert(sizeof(Ctrl) <= 256, "control block must fit 256 bytes");

constexpr int32_t kStatusNonFinite = 1 << 4;   // (1 << WENOZN_ENONFINITE)

// Largest |u_n| + c of one conserved state, with the operation order of the oracle and no
// contraction (so the global maximum, a pure comparison, is bit-identical to it).
// Returns false when the state is not admissible (non-finite, rho <= 0 or p <= 0).
template <int NV>
__device__ __forceinline__ bool wave_state(const double* s, double gamma, double& u, double& v, double& c) {
    const double rho = s[0];
    u = __ddiv_rn(s[1], rho);
    v = NV == 4 ? __ddiv_rn(s[2], rho) : 0.0;
    const double E = s[NV - 1];
    double kin;
    if (NV == 4) kin = __dmul_rn(__dmul_rn(0.5, rho), __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)));
    else kin = __dmul_rn(__dmul_rn(__dmul_rn(0.5, rho), u), u);
    const double p = __dmul_rn(__dadd_rn(gamma, -1.0), __dadd_rn(E, -kin));
    c = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), rho));
    return rho > 0.0 && p > 0.0 && isfinite(E);
}

template <int NV>
__device__ __forceinline__ bool wave_speeds(const double* s, double gamma, double& sx, double& sy) {
    double u, v, c;
    const bool adm = wave_state<NV>(s, gamma, u, v, c);
    sx = __dadd_rn(fabs(u), c);
    sy = NV == 4 ? __dadd_rn(fabs(v), c) : 0.0;
    return adm && isfinite(sx) && isfinite(sy);
}

// Per-field speeds |u-c|, |u|, |u+c| of one direction (the oracle's operation order).
__device__ __forceinline__ void field_speeds(double u, double c, double* f) {
    f[0] = fabs(__dadd_rn(u, -c));
    f[1] = fabs(u);
    f[2] = fabs(__dadd_rn(u, c));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide maximum of two non-negative values, folded into dst[0] and dst[1] (bit-pattern
// atomicMax: order-independent and exact); with only_first, just vx into dst[0].  Must be
// called by every thread of the block.
__device__ __forceinline__ void block_max2_atomic(double vx, double vy, unsigned long long* dst,
                                                  bool only_first = false) {
    __shared__ double red[2][32];
    vx = warp_max(vx);
    vy = warp_max(vy);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) { red[0][w] = vx; red[1][w] = vy; }
    __syncthreads();
    if (w == 0) {
        vx = lane < nw ? red[0][lane] : 0.0;
        vy = lane < nw ? red[1][lane] : 0.0;
        vx = warp_max(vx);
        vy = warp_max(vy);
        if (lane == 0) {
            atomicMax(&dst[0], (unsigned long long)__double_as_longlong(vx));
            if (!only_first) atomicMax(&dst[1], (unsigned long long)__double_as_longlong(vy));
        }
    }
}

// Block-wide maxima of N non-negative values folded into dst[0..N-1] (bit-pattern
// atomicMax).  Must be called by every thread of the block.
template <int N>
__device__ __forceinline__ void block_max_n_atomic(const double* v, unsigned long long* dst) {
    __shared__ double red[N][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const double m = warp_max(v[k]);
        if (lane == 0) red[k][w] = m;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const double m = warp_max(lane < nw ? red[k][lane] : 0.0);
            if (lane == 0) atomicMax(&dst[k], (unsigned long long)__double_as_longlong(m));
        }
    }
    __syncthreads();
}

// Programmatic dependent launch: kernels launched with launch_pdl may start while the
// previous kernel in the stream finishes.  Each of them first waits here for that kernel's
// completion (and memory), before touching anything, then lets its own dependents be
// scheduled.  Without a programmatic dependency both instructions return at once.
__device__ __forceinline__ void pdl_wait() {
#ifdef __CUDA_ARCH__
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// Ghost-cell index map: periodic wrap (bc 0), zero-order extrapolation (outflow, bc 1), or
// the mirror image across the wall (reflective, bc 2: cell -1-g for g < 0, 2n-1-g for
// g >= n, repeated for tiny grids, i.e. the grid continued with period 2n and mirrored in
// every other copy).
__host__ __device__ __forceinline__ int ghost_src(int g, int n, int bc) {
    if (bc == 0) {
        g %= n;
        return g < 0 ? g + n : g;
    }
    if (bc == 2) {
        int m = g % (2 * n);
        if (m < 0) m += 2 * n;
        return m < n ? m : 2 * n - 1 - m;
    }
    return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

// Whether the reflective ghost g is a mirror image (its normal momentum changes sign).
__host__ __device__ __forceinline__ bool ghost_mirrored(int g, int n, int bc) {
    if (bc != 2) return false;
    int m = g % (2 * n);
    if (m < 0) m += 2 * n;
    return m >= n;
}

}  // namespace wz
