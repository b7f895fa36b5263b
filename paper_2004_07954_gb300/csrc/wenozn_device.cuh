// Device-side building blocks of the WENO-ZN solver (FP64, sm_103a).
//
// The arithmetic here is the paper's, rearranged for a GPU whose FP64 pipe is the scarce
// resource: constants are folded, the three un-normalised weights are brought to a common
// denominator so that one division per reconstruction remains, and comparisons of
// non-negative indicators run on the integer pipe.  Every rearrangement is exact algebra;
// only the rounding differs from the plain evaluation order.
#pragma once

#include <cstdint>

namespace wz {

// ------------------------------------------------------------------------------------
// Fifth-order WENO-ZN reconstruction f^+_{i+1/2} from (a, b, c, d, e) = f_{i-2 .. i+2}.
//
//   Eq. (4)        q_0 = (2a - 7b + 11c)/6, q_1 = (-b + 5c + 2d)/6, q_2 = (2c + 5d - e)/6
//   Eq. (isjiang)  IS_k = 13/12 s_k^2 + 1/4 t_k^2 with s_k the second difference and t_k
//                  the one-sided first differences of sub-stencil k
//   Eq. (tau)      tau5 = |IS_0 - IS_2|
//   Eq. (tau8)     tau8 = (a - 4b + 6c - 4d + e)^2
//   Eq. (function) C = A ((IS_0 + IS_2 - tau5 + eps)/(tau5 + eps))^2
//   Eq. (new)      alpha_k = c_k (C + tau8/(IS_k + eps)),  c = (1, 6, 3)/10
//   Eq. (3)        f^ = sum_k alpha_k q_k / sum_k alpha_k
//
// Evaluation: indicators and tau8 are carried scaled by 4 (4 IS_k = 13/3 s_k^2 + t_k^2,
// 4 tau8 = (2 d4)^2) with eps4 = 4 eps, which leaves C and tau8/(IS_k + eps) unchanged.
// IS_0 + IS_2 - tau5 = 2 min(IS_0, IS_2).  Multiplying every alpha_k by
// (tau5 + eps)^2 (IS_0 + eps)(IS_1 + eps)(IS_2 + eps) / c_k gives
//   a_k = A m^2 b_0 b_1 b_2 + 4 tau8 P^2 prod_{j != k} b_j,  m = 2 min + eps, P = tau5 + eps,
// all positive (a_k >= A (4 eps)^5 > 0), and the optimal weights are folded into the
// integer coefficients of the sub-stencil fluxes.  Range: finite for |f| below ~1e20.
// ------------------------------------------------------------------------------------
struct ZnParts {
    double num, den;     // f^ = num / den
};

__device__ __forceinline__ ZnParts zn_parts(double a, double b, double c, double d, double e,
                                            double eps4, double A) {
    const double s0 = fma(-2.0, b, a) + c;
    const double s1 = fma(-2.0, c, b) + d;
    const double s2 = fma(-2.0, d, c) + e;
    const double t0 = fma(3.0, c, fma(-4.0, b, a));
    const double t1 = b - d;
    const double t2 = fma(3.0, c, fma(-4.0, d, e));
    const double k13_3 = 13.0 / 3.0;
    const double is0 = fma(k13_3 * s0, s0, t0 * t0);
    const double is1 = fma(k13_3 * s1, s1, t1 * t1);
    const double is2 = fma(k13_3 * s2, s2, t2 * t2);
    const double d4 = fma(-2.0, s1, s0) + s2;               // fourth difference
    // non-negative doubles order like their bit patterns: min/max on the integer pipe
    const long long i0 = __double_as_longlong(is0), i2 = __double_as_longlong(is2);
    const double mn = __longlong_as_double(i0 < i2 ? i0 : i2);
    const double mx = __longlong_as_double(i0 < i2 ? i2 : i0);
    const double P = (mx - mn) + eps4;                       // tau5 + eps
    const double m = fma(2.0, mn, eps4);                     // IS_0 + IS_2 - tau5 + eps
    const double b0 = is0 + eps4, b1 = is1 + eps4, b2 = is2 + eps4;
    const double b01 = b0 * b1, b12 = b1 * b2, b02 = b0 * b2;
    const double X = (A * m) * m * (b01 * b2);
    const double z = d4 * P;
    const double Y = 4.0 * (z * z);
    const double a0 = fma(Y, b12, X), a1 = fma(Y, b02, X), a2 = fma(Y, b01, X);
    const double q0 = fma(11.0, c, fma(-7.0, b, 2.0 * a));   //  6 q_0
    const double q1 = fma(12.0, d, fma(30.0, c, -6.0 * b));  // 36 q_1
    const double q2 = fma(15.0, d, fma(6.0, c, -3.0 * e));   // 18 q_2
    ZnParts r;
    r.num = fma(a0, q0, fma(a1, q1, a2 * q2));
    r.den = fma(6.0, a0, fma(36.0, a1, 18.0 * a2));
    return r;
}

__device__ __forceinline__ double zn_flux(double a, double b, double c, double d, double e,
                                          double eps4, double A) {
    const ZnParts r = zn_parts(a, b, c, d, e, eps4, A);
    return r.num / r.den;
}

// f^+ + f^- at one interface: plus side from (p0..p4) = h+_{i-2..i+2}, minus side from the
// mirrored stencil (m4, m3, m2, m1, m0) where (m0..m4) = h-_{i-1..i+3} (Sec. 2, the
// "symmetric rule about x_{i+1/2}").
__device__ __forceinline__ double zn_split_flux(double p0, double p1, double p2, double p3, double p4,
                                                double m0, double m1, double m2, double m3, double m4,
                                                double eps4, double A) {
    return zn_flux(p0, p1, p2, p3, p4, eps4, A) + zn_flux(m4, m3, m2, m1, m0, eps4, A);
}

// ------------------------------------------------------------------------------------
// Workspace control block (first 256 bytes of the caller's workspace).
// ------------------------------------------------------------------------------------
struct Ctrl {
    unsigned long long alpha[3][2];   // LF speeds per RK stage slot, as IEEE bit patterns
    double dt;                        // the step the current RK3 step uses
    int32_t status;                   // OR of (1 << wenozn_status) device-detected bits
    int32_t pad0;
    double reserved[24];
};
static_assert(sizeof(Ctrl) <= 256, "control block must fit 256 bytes");

constexpr int32_t kStatusNonFinite = 1 << 4;   // (1 << WENOZN_ENONFINITE)

// Largest |u_n| + c of one conserved state, with the operation order of the oracle and no
// contraction (so the global maximum, a pure comparison, is bit-identical to it).
// Returns false when the state is not admissible (non-finite, rho <= 0 or p <= 0).
template <int NV>
__device__ __forceinline__ bool wave_speeds(const double* s, double gamma, double& sx, double& sy) {
    const double rho = s[0];
    const double u = __ddiv_rn(s[1], rho);
    const double v = NV == 4 ? __ddiv_rn(s[2], rho) : 0.0;
    const double E = s[NV - 1];
    double kin;
    if (NV == 4) kin = __dmul_rn(__dmul_rn(0.5, rho), __dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)));
    else kin = __dmul_rn(__dmul_rn(__dmul_rn(0.5, rho), u), u);
    const double p = __dmul_rn(__dadd_rn(gamma, -1.0), __dadd_rn(E, -kin));
    const double c = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), rho));
    sx = __dadd_rn(fabs(u), c);
    sy = NV == 4 ? __dadd_rn(fabs(v), c) : 0.0;
    const bool ok = rho > 0.0 && p > 0.0 && isfinite(sx) && isfinite(sy) && isfinite(E);
    return ok;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide maximum of two non-negative values, folded into `dst` (bit-pattern atomicMax:
// order-independent and exact).  Must be called by every thread of the block.
__device__ __forceinline__ void block_max2_atomic(double vx, double vy, unsigned long long* dst) {
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
            atomicMax(&dst[1], (unsigned long long)__double_as_longlong(vy));
        }
    }
}

// Ghost-cell index map: periodic wrap or zero-order extrapolation (outflow).
__device__ __forceinline__ int ghost_src(int g, int n, int bc) {
    if (bc == 0) {
        g %= n;
        return g < 0 ? g + n : g;
    }
    return g < 0 ? 0 : (g >= n ? n - 1 : g);
}

}  // namespace wz
