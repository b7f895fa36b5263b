// Discrete adjoint (vector-Jacobian products) of the 1D right-hand side and of the SSP-RK3
// step, written by hand from the forward arithmetic.
//
// RHS: L_i = -(F^_{i+1/2} - F^_{i-1/2})/dx, F^ at interface j (x_{j-1/2}) depends on the six
// cells j-3 .. j+2 and on the global LF speed alpha = max_i(|u_i| + c_i).  For a cotangent
// lambda of L the interface cotangent is Fbar_j = (lambda_j - lambda_{j-1})/dx (lambda outside
// the grid is 0).  Each interface thread recomputes its forward quantities and sweeps them
// backwards, writing the cotangent contributions to its six stencil cells into a buffer
// C[j][s][k]; a gather kernel then sums, for every cell, the contributions of the stencil
// positions that map to it (ghost cells included) in a fixed order, so the result is
// deterministic.  alpha is differentiated through its argmax cell (the lowest index on ties);
// d|x|/dx is taken as 0 at x = 0.
#include "launch.h"

namespace wz {

namespace {

constexpr int kThreads = 128;

// Reverse of zn_flux: given f[0..4] and the cotangent Wb of f^ = W(f), adds dW/df * Wb to fb.
__host__ __device__ __forceinline__ void zn_vjp(const double* f, double Wb, double eps4, double A4, double* fb) {
    const double a = f[0], b = f[1], c = f[2], d = f[3], e = f[4];
    // first differences, then the second (s_k) and one-sided (t_k) differences from them:
    // equal inputs give exact zeros
    const double D1 = a - b, D2 = b - c, D3 = c - d, D4 = d - e;
    const double s0 = D1 - D2, s1 = D2 - D3, s2 = D3 - D4;
    const double t0 = fma(-3.0, D2, D1), t1 = D2 + D3, t2 = fma(3.0, D3, -D4);
    const double k13_3 = 13.0 / 3.0;
    const double b0 = fma(k13_3 * s0, s0, fma(t0, t0, eps4));
    const double b1 = fma(k13_3 * s1, s1, fma(t1, t1, eps4));
    const double b2 = fma(k13_3 * s2, s2, fma(t2, t2, eps4));
    const double d4 = t0 + t2;
    const double sg = b0 > b2 ? 1.0 : (b0 < b2 ? -1.0 : 0.0);   // sign(IS_0 - IS_2), 0 on ties
    const double mn = fmin(b0, b2), mx = fmax(b0, b2);
    const double P = (mx - mn) + eps4;
    const double m = fma(2.0, mn, -eps4);
    const double b12 = b1 * b2, b02 = b0 * b2, b01 = b0 * b1;
    const double K = (A4 * m) * m;
    const double X = K * (b01 * b2);
    const double z = d4 * P;
    const double Y = z * z;
    const double a0 = fma(Y, b12, X), a1 = fma(Y, b02, X), a2 = fma(Y, b01, X);
    const double q0 = fma(1.0 / 12.0, s0, fma(0.25, t0, c));
    const double q1 = fma(0.5, s1, fma(-1.5, t1, 6.0 * c));
    const double q2 = fma(0.25, s2, fma(-0.75, t2, 3.0 * c));
    const double N = fma(a0, q0, fma(a1, q1, a2 * q2));
    const double D = fma(6.0, a1, fma(3.0, a2, a0));
    const double rD = 1.0 / D;
    const double W = N * rD;
    // reverse
    const double Nb = Wb * rD, Db = -Wb * W * rD;
    const double a0b = fma(Nb, q0, Db), a1b = fma(Nb, q1, 6.0 * Db), a2b = fma(Nb, q2, 3.0 * Db);
    const double q0b = Nb * a0, q1b = Nb * a1, q2b = Nb * a2;
    const double Xb = a0b + a1b + a2b;
    const double Yb = fma(a0b, b12, fma(a1b, b02, a2b * b01));
    const double XK = Xb * K;
    double b0b = fma(Y, fma(a1b, b2, a2b * b1), XK * b12);
    double b1b = fma(Y, fma(a0b, b2, a2b * b0), XK * b02);
    double b2b = fma(Y, fma(a0b, b1, a1b * b0), XK * b01);
    const double mb = Xb * (b01 * b2) * (2.0 * A4 * m);
    const double zb = 2.0 * z * Yb;
    const double d4b = zb * P, Pb = zb * d4;
    const double taub = Pb - mb;                    // P = tau + eps4, m = b0 + b2 - tau - eps4
    b0b += mb + sg * taub;
    b2b += mb - sg * taub;
    double s0b = b0b * (2.0 * k13_3) * s0, s1b = b1b * (2.0 * k13_3) * s1, s2b = b2b * (2.0 * k13_3) * s2;
    double t0b = b0b * 2.0 * t0 + d4b, t1b = b1b * 2.0 * t1, t2b = b2b * 2.0 * t2 + d4b;
    const double cb = q0b + 6.0 * q1b + 3.0 * q2b;
    s0b += q0b / 12.0;
    t0b += 0.25 * q0b;
    s1b += 0.5 * q1b;
    t1b -= 1.5 * q1b;
    s2b += 0.25 * q2b;
    t2b -= 0.75 * q2b;
    fb[0] += s0b + t0b;
    fb[1] += -2.0 * s0b + s1b - 4.0 * t0b + t1b;
    fb[2] += cb + s0b - 2.0 * s1b + s2b + 3.0 * t0b + 3.0 * t2b;
    fb[3] += s1b - 2.0 * s2b - t1b - 4.0 * t2b;
    fb[4] += s2b + t2b;
}

// Cotangents Ub[6][NV] of the six stencil cells (and alpha) of one interface flux, given
// the cotangent Fb of F^ at that interface.  NV = 1: advection with speed a (alpha = |a|,
// constant); NV = 3: 1D Euler.
template <int NV>
__host__ __device__ void interface_vjp(const double (*Us)[3], double alpha, double a_adv, double gamma, double eps4,
                              double A4, const double* Fb, double (*Ub)[3], double& alphab) {
    const double gm1 = gamma - 1.0;
    double hp[6][NV], hm[6][NV];
    double u[6], p[6], Ep[6];
    for (int s = 0; s < 6; ++s) {
        if (NV == 1) {
            const double f = a_adv * Us[s][0];
            hp[s][0] = 0.5 * (f + alpha * Us[s][0]);
            hm[s][0] = 0.5 * (f - alpha * Us[s][0]);
            continue;
        }
        const double rho = Us[s][0], mom = Us[s][1], E = Us[s][2];
        u[s] = mom / rho;
        p[s] = gm1 * (E - 0.5 * mom * u[s]);
        Ep[s] = E + p[s];
        const double F[3] = {mom, fma(mom, u[s], p[s]), u[s] * Ep[s]};
        for (int k = 0; k < 3; ++k) {
            hp[s][k] = 0.5 * (F[k] + alpha * Us[s][k]);
            hm[s][k] = 0.5 * (F[k] - alpha * Us[s][k]);
        }
    }
    for (int s = 0; s < 6; ++s)
        for (int k = 0; k < 3; ++k) Ub[s][k] = 0.0;
    alphab = 0.0;
    double hpb[6][NV], hmb[6][NV];
    for (int s = 0; s < 6; ++s)
        for (int k = 0; k < NV; ++k) hpb[s][k] = hmb[s][k] = 0.0;

    if (NV == 1) {
        const double fp[5] = {hp[0][0], hp[1][0], hp[2][0], hp[3][0], hp[4][0]};
        const double fm[5] = {hm[5][0], hm[4][0], hm[3][0], hm[2][0], hm[1][0]};
        double fpb[5] = {0, 0, 0, 0, 0}, fmb[5] = {0, 0, 0, 0, 0};
        zn_vjp(fp, Fb[0], eps4, A4, fpb);
        zn_vjp(fm, Fb[0], eps4, A4, fmb);
        for (int s = 0; s < 5; ++s) {
            hpb[s][0] += fpb[s];
            hmb[5 - s][0] += fmb[s];
        }
        for (int s = 0; s < 6; ++s)
            Ub[s][0] = 0.5 * (a_adv + alpha) * hpb[s][0] + 0.5 * (a_adv - alpha) * hmb[s][0];
        return;
    }

    // ---- forward: Roe state and eigenvectors of cells 2 and 3 ----------------------------
    const double rhoL = Us[2][0], rhoR = Us[3][0];
    const double sl = sqrt(rhoL), sr = sqrt(rhoR);
    const double HL = Ep[2] / rhoL, HR = Ep[3] / rhoR;
    const double S = sl + sr;
    const double wl = sl / S, wr = sr / S;
    const double ut = wl * u[2] + wr * u[3];
    const double Ht = wl * HL + wr * HR;
    const double c2 = gm1 * (Ht - 0.5 * ut * ut);
    const double c = sqrt(c2);
    const double rc = 1.0 / c;
    const double b1 = gm1 * rc * rc, b2 = 0.5 * ut * ut * b1;
    const double Lm[3][3] = {{0.5 * (b2 + ut * rc), -0.5 * (b1 * ut + rc), 0.5 * b1},
                             {1.0 - b2, b1 * ut, -b1},
                             {0.5 * (b2 - ut * rc), -0.5 * (b1 * ut - rc), 0.5 * b1}};
    const double R[3][3] = {{1.0, 1.0, 1.0},
                            {ut - c, ut, ut + c},
                            {Ht - ut * c, 0.5 * ut * ut, Ht + ut * c}};
    double gp[3][5], gm[3][5], gh[3];
    for (int k = 0; k < 3; ++k) {
        for (int s = 0; s < 5; ++s) {
            gp[k][s] = Lm[k][0] * hp[s][0] + Lm[k][1] * hp[s][1] + Lm[k][2] * hp[s][2];
            gm[k][s] = Lm[k][0] * hm[s + 1][0] + Lm[k][1] * hm[s + 1][1] + Lm[k][2] * hm[s + 1][2];
        }
        const double fpk[5] = {gp[k][0], gp[k][1], gp[k][2], gp[k][3], gp[k][4]};
        const double fmk[5] = {gm[k][4], gm[k][3], gm[k][2], gm[k][1], gm[k][0]};
        gh[k] = zn_flux(fpk[0], fpk[1], fpk[2], fpk[3], fpk[4], eps4, A4, false) +
                zn_flux(fmk[0], fmk[1], fmk[2], fmk[3], fmk[4], eps4, A4, false);
    }
    // ---- reverse --------------------------------------------------------------------------
    double ghb[3], Rb[3][3], Lb[3][3];
    for (int k = 0; k < 3; ++k) {
        ghb[k] = R[0][k] * Fb[0] + R[1][k] * Fb[1] + R[2][k] * Fb[2];
        for (int m = 0; m < 3; ++m) {
            Rb[m][k] = Fb[m] * gh[k];
            Lb[k][m] = 0.0;
        }
    }
    for (int k = 0; k < 3; ++k) {
        const double fpk[5] = {gp[k][0], gp[k][1], gp[k][2], gp[k][3], gp[k][4]};
        const double fmk[5] = {gm[k][4], gm[k][3], gm[k][2], gm[k][1], gm[k][0]};
        double fpb[5] = {0, 0, 0, 0, 0}, fmb[5] = {0, 0, 0, 0, 0};
        zn_vjp(fpk, ghb[k], eps4, A4, fpb);
        zn_vjp(fmk, ghb[k], eps4, A4, fmb);
        for (int s = 0; s < 5; ++s) {
            const double gpb = fpb[s], gmb = fmb[4 - s];       // cotangents of gp[k][s], gm[k][s]
            for (int m = 0; m < 3; ++m) {
                Lb[k][m] += gpb * hp[s][m] + gmb * hm[s + 1][m];
                hpb[s][m] += gpb * Lm[k][m];
                hmb[s + 1][m] += gmb * Lm[k][m];
            }
        }
    }
    // left eigenvectors -> (u~, rc, b1, b2)
    double b2b = 0.5 * Lb[0][0] - Lb[1][0] + 0.5 * Lb[2][0];
    double b1b = -0.5 * ut * Lb[0][1] + 0.5 * Lb[0][2] + ut * Lb[1][1] - Lb[1][2] - 0.5 * ut * Lb[2][1] +
                 0.5 * Lb[2][2];
    double rcb = 0.5 * ut * Lb[0][0] - 0.5 * Lb[0][1] - 0.5 * ut * Lb[2][0] + 0.5 * Lb[2][1];
    double utb = 0.5 * rc * Lb[0][0] - 0.5 * b1 * Lb[0][1] + b1 * Lb[1][1] - 0.5 * rc * Lb[2][0] -
                 0.5 * b1 * Lb[2][1];
    utb += b2b * ut * b1;
    b1b += b2b * 0.5 * ut * ut;
    rcb += b1b * 2.0 * gm1 * rc;
    double cb = -rcb * rc * rc;
    // right eigenvectors -> (u~, c, H~)
    utb += Rb[1][0] + Rb[1][1] + Rb[1][2] - c * Rb[2][0] + ut * Rb[2][1] + c * Rb[2][2];
    cb += -Rb[1][0] + Rb[1][2] - ut * Rb[2][0] + ut * Rb[2][2];
    double Htb = Rb[2][0] + Rb[2][2];
    // c = sqrt((gamma-1)(H~ - u~^2/2))
    Htb += cb * gm1 * 0.5 * rc;
    utb -= cb * gm1 * 0.5 * rc * ut;
    // Roe average -> u, H of cells 2 and 3 and sqrt(rho)
    double ub[6] = {0, 0, 0, 0, 0, 0}, Hb2 = Htb * wl, Hb3 = Htb * wr;
    ub[2] += utb * wl;
    ub[3] += utb * wr;
    const double slb = (utb * (u[2] - ut) + Htb * (HL - Ht)) / S;
    const double srb = (utb * (u[3] - ut) + Htb * (HR - Ht)) / S;
    Ub[2][0] += slb * 0.5 / sl;
    Ub[3][0] += srb * 0.5 / sr;
    // cells: split fluxes, enthalpy, primitives
    for (int s = 0; s < 6; ++s) {
        const double rho = Us[s][0], mom = Us[s][1];
        double Fbc[3], pb = 0.0;
        for (int k = 0; k < 3; ++k) {
            Fbc[k] = 0.5 * (hpb[s][k] + hmb[s][k]);
            const double dh = 0.5 * (hpb[s][k] - hmb[s][k]);
            Ub[s][k] += alpha * dh;
            alphab += Us[s][k] * dh;
        }
        double mb = Fbc[0] + Fbc[1] * u[s];
        double Eb = Fbc[2] * u[s];
        ub[s] += Fbc[1] * mom + Fbc[2] * Ep[s];
        pb += Fbc[1] + Fbc[2] * u[s];
        if (s == 2 || s == 3) {
            const double Hb = s == 2 ? Hb2 : Hb3;
            Eb += Hb / rho;
            pb += Hb / rho;
            Ub[s][0] -= Hb * (Ep[s] / rho) / rho;
        }
        Eb += gm1 * pb;
        mb -= gm1 * 0.5 * u[s] * pb;
        ub[s] -= gm1 * 0.5 * mom * pb;
        mb += ub[s] / rho;
        Ub[s][0] -= ub[s] * u[s] / rho;
        Ub[s][1] += mb;
        Ub[s][2] += Eb;
    }
}

// Per interface: cotangent contributions to its six stencil cells (C[j][s][k]) and a
// per-block partial sum of the LF-speed cotangent.
template <int NV>
__global__ void __launch_bounds__(kThreads) vjp_interface_kernel(VjpArgs a) {
    __shared__ double red[kThreads / 32];
    const int n = a.n;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    double alphab = 0.0;
    if (j <= n) {
        double Us[6][3];
        for (int s = 0; s < 6; ++s) {
            const int g = ghost_src(j - 3 + s, n, a.bc);
            for (int k = 0; k < NV; ++k) Us[s][k] = a.U[int64_t(k) * n + g];
        }
        double Fb[NV];
        for (int k = 0; k < NV; ++k) {
            const double right = j < n ? a.lam[int64_t(k) * n + j] : 0.0;
            const double left = j > 0 ? a.lam[int64_t(k) * n + j - 1] : 0.0;
            Fb[k] = (right - left) * a.rdx;
        }
        const double alpha = NV == 1 ? fabs(a.adv_speed) : __longlong_as_double((long long)a.alpha_bits[0]);
        double Ub[6][3];
        interface_vjp<NV>(Us, alpha, a.adv_speed, a.gamma, a.eps4, a.A4, Fb, Ub, alphab);
        double* out = a.C + int64_t(j) * 6 * NV;
        for (int s = 0; s < 6; ++s)
            for (int k = 0; k < NV; ++k) out[s * NV + k] = Ub[s][k];
    }
    // deterministic per-block partial of the LF-speed cotangent
    double v = alphab;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        a.partial[blockIdx.x] = t;
    }
}

// Lowest cell index whose |u| + c equals the LF speed (bit-exact comparison).
template <int NV>
__global__ void __launch_bounds__(256) argmax_kernel(VjpArgs a) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= a.n || NV == 1) return;
    double s[NV];
    for (int k = 0; k < NV; ++k) s[k] = a.U[int64_t(k) * a.n + i];
    double sx, sy;
    wave_speeds<NV>(s, a.gamma, sx, sy);
    if (__double_as_longlong(sx) == (long long)a.alpha_bits[0]) atomicMin(a.argmax, i);
}

// out_i = c1 X1_i + c2 X2_i + c3 X3_i + d (J^T lambda)_i with the gathered contributions.
template <int NV>
__global__ void __launch_bounds__(256) vjp_gather_kernel(VjpArgs a) {
    const int n = a.n;
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    double acc[NV];
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    // stencil cells g (in -3 .. n+2) whose ghost map lands on i
    int gs[16], ng = 0;
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
            const int j = g + 3 - s;                 // interface whose stencil position s is g
            if (j < 0 || j > n) continue;
            const double* c = a.C + (int64_t(j) * 6 + s) * NV;
            for (int k = 0; k < NV; ++k) acc[k] += c[k];
        }
    }
    if (NV == 3 && i == *a.argmax) {
        double ab = 0.0;
        for (int b = 0; b < a.nblocks; ++b) ab += a.partial[b];
        // d(|u| + c)/dU at this cell, |x|' = 0 at 0
        const double rho = a.U[i], mom = a.U[n + i], E = a.U[2 * int64_t(n) + i];
        const double u = mom / rho;
        const double p = (a.gamma - 1.0) * (E - 0.5 * mom * u);
        const double c = sqrt(a.gamma * p / rho);
        const double sg = u > 0.0 ? 1.0 : (u < 0.0 ? -1.0 : 0.0);
        const double k = a.gamma / (2.0 * c * rho), gm1 = a.gamma - 1.0;
        acc[0] += ab * (sg * (-u / rho) + k * (gm1 * 0.5 * u * u - p / rho));
        acc[1] += ab * (sg / rho - k * gm1 * u);
        acc[2] += ab * (k * gm1);
    }
    for (int k = 0; k < NV; ++k) {
        const int64_t idx = int64_t(k) * n + i;
        double r = a.d * acc[k];
        if (a.X1) r = fma(a.c1, a.X1[idx], r);
        if (a.X2) r = fma(a.c2, a.X2[idx], r);
        if (a.X3) r = fma(a.c3, a.X3[idx], r);
        a.out[idx] = r;
    }
}

}  // namespace

int vjp_interface_blocks(int n) { return (n + 1 + kThreads - 1) / kThreads; }

cudaError_t launch_vjp(int system, const VjpArgs& a, cudaStream_t s) {
    const unsigned gi = unsigned(vjp_interface_blocks(a.n)), gc = unsigned((a.n + 255) / 256);
    if (system == 0) {
        vjp_interface_kernel<1><<<gi, kThreads, 0, s>>>(a);
        vjp_gather_kernel<1><<<gc, 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(a.argmax, 0x7f, sizeof(int), s);   // a large positive int
    if (e != cudaSuccess) return e;
    argmax_kernel<3><<<gc, 256, 0, s>>>(a);
    vjp_interface_kernel<3><<<gi, kThreads, 0, s>>>(a);
    vjp_gather_kernel<3><<<gc, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace wz
