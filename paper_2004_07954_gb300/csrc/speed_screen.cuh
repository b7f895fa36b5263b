// Screening of the LF-speed maximum (Sec. 2: alpha = max |u_n| + c over the grid).
//
// The maximum has to be bit-identical to a plain IEEE evaluation in the oracle's operation
// order, whose two or three divisions and one square root cost about 45 FP64 instructions
// per cell.  Only the cell that attains the maximum needs that exact value, so every cell
// first gets a single-precision estimate with a proven error bound, and the exact value is
// evaluated only where the estimate comes within a relative window tau of the running
// maximum of the estimates (or where no bound is available).
//
// Estimate.  For rho, E in [2^-30, 2^30), |m| < 2^30 (|m| < 2^-100 taken as 0) every input
// becomes a float by keeping sign, exponent and the leading 20 fraction bits of the double
// (integer operations; relative truncation error below 2^-20).  Then, in float with IEEE
// rounding (unit roundoff 2^-24):
//   r = 1/rho, u = m r, e = E - (m u [+ n v])/2, c = sqrt(gamma (gamma-1) e r), s = |u| + c.
// The estimate is used only when e >= E/8 (the internal energy is at least an eighth of the
// total, i.e. Mach number up to 5 for gamma = 1.4); then
//   * u carries at most 2.1 * 2^-20 relative error, the kinetic part 3.2 * 2^-20, so e is
//     within 4.3 * 2^-20 E <= 34.4 * 2^-20 e of its exact value;
//   * c^2 within 36.6 * 2^-20, c within 18.3 * 2^-20, s within 18.4 * 2^-20 < 1.8e-5 relative;
//   * the FP64 evaluation itself is within 1e-14 relative of the exact speed (its
//     cancellation in E - kin is bounded by the same e >= E/8),
// so |s_est - s_exact| <= delta s_exact with delta = 1.8e-5.
//
// Window.  Let j attain the maximum of the exact speeds over a set of cells and M the
// maximum of the estimates over the screened cells of that set processed so far (j's own
// batch included).  Then M <= (1 + delta) s(j) and s_est(j) >= (1 - delta) s(j), so
// s_est(j) >= M (1 - delta)/(1 + delta) >= M (1 - tau) for tau >= 2 delta / (1 - delta):
// j is always evaluated exactly, and the maximum over the exactly evaluated cells is the
// exact maximum.  tau = 2^-11 = 4.9e-4 leaves a factor 13 over 2 delta.  Cells passed over
// are admissible (rho > 0, p > 0, finite), so the status word is unaffected.
#pragma once

#include <cstdint>

namespace wz {

constexpr float kScreenKeep = 1.0f - 1.0f / 2048.0f;   // 1 - tau

// float with the sign, exponent and leading 20 fraction bits of the double whose high word
// is hi; valid for magnitudes in [2^-126, 2^128)
__device__ __forceinline__ float f32_trunc_hi(int hi) {
    const unsigned h = unsigned(hi);
    return __uint_as_float((((h & 0x7fffffffu) - (896u << 20)) << 3) | (h & 0x80000000u));
}

__device__ __forceinline__ bool positive_in_range(int hi) {          // 2^-30 <= x < 2^30
    return unsigned(hi) - (993u << 20) < (60u << 20);
}

// momentum component: |m| < 2^30 required; |m| < 2^-100 taken as 0
__device__ __forceinline__ float momentum_f32(int hi, bool& ok) {
    const int mag = hi & 0x7fffffff;
    ok = ok && mag < (1053 << 20);
    return mag < (923 << 20) ? 0.0f : f32_trunc_hi(hi);
}

struct SpeedEstimate {
    float sx, sy;   // estimates of |u| + c and |v| + c (0 where not ok)
    float u, v, c;  // the estimates they come from (meaningful where ok)
    bool ok;        // the bound of the header holds for this cell
};

// s = (rho, m_x[, m_y], E); gg1 = gamma (gamma - 1) rounded to float
template <int NV>
__device__ __forceinline__ SpeedEstimate estimate_speeds(const double* s, float gg1) {
    const int hr = __double2hiint(s[0]), he = __double2hiint(s[NV - 1]);
    bool ok = positive_in_range(hr) && positive_in_range(he);
    const float rho = f32_trunc_hi(hr), E = f32_trunc_hi(he);
    const float m = momentum_f32(__double2hiint(s[1]), ok);
    const float n = NV == 4 ? momentum_f32(__double2hiint(s[2]), ok) : 0.0f;
    const float r = __frcp_rn(rho);
    const float u = __fmul_rn(m, r);
    const float v = __fmul_rn(n, r);
    const float kin = __fmul_rn(0.5f, __fadd_rn(__fmul_rn(m, u), __fmul_rn(n, v)));
    const float e = __fsub_rn(E, kin);
    ok = ok && e >= __fmul_rn(0.125f, E);
    const float c = __fsqrt_rn(__fmul_rn(__fmul_rn(gg1, e), r));
    SpeedEstimate est;
    est.ok = ok;
    est.sx = ok ? __fadd_rn(fabsf(u), c) : 0.0f;
    est.sy = ok && NV == 4 ? __fadd_rn(fabsf(v), c) : 0.0f;
    est.u = u;
    est.v = v;
    est.c = c;
    return est;
}

// Per-field speeds |u - c|, |u|, |u + c| (and with v in 2D).  Where the estimate is ok, each
// is within delta (|u| + c) (delta = 1.8e-5, as above) of the FP64 value: u and c carry at most
// that relative error and the two subtractions round once each.  So against the running
// maximum M_k of such estimates, the cell attaining the exact maximum of field k always lies
// within 2 delta S of M_k, S the largest |u| + c (|v| + c) of the cells seen; the screen's
// window for the fields is tau max(M_x, M_y) >= 2 delta S.
template <int NV>
__device__ __forceinline__ void estimate_field_speeds(const SpeedEstimate& e, float* f) {
    f[0] = e.ok ? fabsf(__fsub_rn(e.u, e.c)) : 0.0f;
    f[1] = e.ok ? fabsf(e.u) : 0.0f;
    f[2] = e.ok ? fabsf(__fadd_rn(e.u, e.c)) : 0.0f;
    f[3] = e.ok && NV == 4 ? fabsf(__fsub_rn(e.v, e.c)) : 0.0f;
    f[4] = e.ok && NV == 4 ? fabsf(e.v) : 0.0f;
    f[5] = e.ok && NV == 4 ? fabsf(__fadd_rn(e.v, e.c)) : 0.0f;
}

__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Running block-wide maxima of N estimates over the batches of T cells a block processes
// (one barrier per batch; two buffers, so a batch's reads never race the next batch's
// writes).  Every thread of the block must call add() the same number of times.
template <int T, int N = 2>
struct ScreenMax {
    float m[N] = {};
    int parity = 0;
    __device__ __forceinline__ void add(const float* e) {
        __shared__ float red[2][N][T / 32];
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int q = 0; q < N; ++q) {
            const float v = warp_max_f(e[q]);
            if (lane == 0) red[parity][q][w] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < T / 32; ++k)
#pragma unroll
            for (int q = 0; q < N; ++q) m[q] = fmaxf(m[q], red[parity][q][k]);
        parity ^= 1;
    }
};

}  // namespace wz
