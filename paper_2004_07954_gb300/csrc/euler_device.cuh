// Per-cell and per-interface building blocks shared by the single-problem flux kernels and
// the batched kernel: LF flux splitting of one cell (Sec. 2, Sec. 4.3) and the numerical
// flux of one interface (Roe average, characteristic projection, WENO-ZN of both split
// parts, back-projection).  Everything lives in shared memory planes of a tile.
#pragma once

#include "wenozn_device.cuh"

namespace wz {

// Shared-memory planes of one tile of NC cells: split fluxes h+ and h- (NV planes each),
// and for the Euler systems sqrt(rho), u_n, H (and u_t in 2D), the differences
// dh+-_c = h+-_c - h+-_{c+1} along the sweep (NV planes each) and, in the generic kernels,
// the cell's |u_n| + c.
template <int NV>
struct CellPlanes {
    static constexpr int kPerCell = NV == 1 ? 2 : 2 * NV + (NV == 4 ? 4 : 3);
    static constexpr int kPerCellDefault = kPerCell + (NV == 1 ? 0 : 2 * NV);   // + dh+, dh-
    static constexpr int kPerCellGeneric = kPerCellDefault + (NV == 1 ? 0 : 1);   // + |u_n| + c
    double* hp;
    double* hm;
    double* sr;
    double* un;
    double* H;
    double* ut;
    double* dp;          // Euler: dh+ and dh-
    double* dm;
    double* sp;          // generic kernels: the cell's |u_n| + c (local LF)
    int NC;
    __device__ __forceinline__ CellPlanes(double* base, int nc) : NC(nc) {
        hp = base;
        hm = hp + NV * nc;
        sr = hm + NV * nc;
        un = sr + nc;
        H = un + nc;
        ut = H + nc;
        dp = base + kPerCell * nc;
        dm = dp + NV * nc;
        sp = base + kPerCellDefault * nc;
    }
};

// The split-flux differences of cell si and its neighbour si + stride along the sweep, once
// per cell: the characteristic projection is linear, so the reconstructions' stencil
// differences are projections of these (no cell difference is formed per interface and field).
template <int NV>
__device__ __forceinline__ void cell_diffs(const CellPlanes<NV>& s, int si, int stride) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        s.dp[k * s.NC + si] = s.hp[k * s.NC + si] - s.hp[k * s.NC + si + stride];
        s.dm[k * s.NC + si] = s.hm[k * s.NC + si] - s.hm[k * s.NC + si + stride];
    }
}

// One cell: Uc = (rho, m_n[, m_t], E) in the sweep direction's frame (or the scalar u with
// the advection speed `a`), alpha the LF speed.  Writes h+- = (F +- alpha U)/2 and the Roe
// ingredients at shared index si.
template <int NV>
__device__ __forceinline__ void split_cell(const double* Uc, double alpha, double a_adv, double gm1,
                                           const CellPlanes<NV>& s, int si) {
    const double half_a = 0.5 * alpha;
    if (NV == 1) {
        const double u = Uc[0];
        const double f = a_adv * u;
        s.hp[si] = 0.5 * fma(alpha, u, f);
        s.hm[si] = 0.5 * fma(-alpha, u, f);
        return;
    }
    const double rho = Uc[0], mn = Uc[1], E = Uc[NV - 1];
    const double mt = NV == 4 ? Uc[2] : 0.0;
    const double rs = rsqrt(rho);
    const double rr = rs * rs;                         // 1 / rho
    const double un = mn * rr;
    const double ut = mt * rr;
    // p/2 = (gamma-1)(E - (m_n u_n + m_t u_t)/2)/2
    const double mq = NV == 4 ? fma(mn, un, mt * ut) : mn * un;
    const double hp2 = fma(-0.25 * gm1, mq, (0.5 * gm1) * E);
    const double Ep = fma(2.0, hp2, E);
    // half the physical flux, F/2 = (m_n, m_n u_n + p, m_t u_n, u_n (E + p)) / 2
    const double hun = 0.5 * un;
    double hF[NV];
    hF[0] = 0.5 * mn;
    hF[1] = fma(mn, hun, hp2);
    if (NV == 4) hF[2] = mt * hun;
    hF[NV - 1] = hun * Ep;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        s.hp[k * s.NC + si] = fma(half_a, Uc[k], hF[k]);
        s.hm[k * s.NC + si] = fma(-half_a, Uc[k], hF[k]);
    }
    s.sr[si] = rho * rs;                               // sqrt(rho)
    s.un[si] = un;
    s.H[si] = Ep * rr;
    if (NV == 4) s.ut[si] = ut;
}

// The cell phase of the generic kernels, by splitting (split: 0 global LF, 1 per-field LF,
// 2 local LF, 3 Steger-Warming):
//   0     h+- = (F +- alpha U)/2, as split_cell;
//   1, 2  hp = F/2, hm = U/2 (split after the projection, per field or per interface), and
//         for 2 the cell's |u_n| + c in the speed plane;
//   3     hp = F+, hm = F- of Steger and Warming:
//         F+- = rho/(2 gamma) (2(g-1) l2 + l1 + l3, 2(g-1) l2 u + l1 (u-c) + l3 (u+c),
//                              [(2(g-1) l2 + l1 + l3) v,] (g-1) l2 q^2 + l1 ((u-c)^2 + v^2)/2
//                              + l3 ((u+c)^2 + v^2)/2 + (3-g)(l1 + l3) c^2 / (2(g-1)))
//         with l = (u-c, u, u+c) and l+- = (l +- |l|)/2, q^2 = u^2 + v^2.
// Advection ignores the splitting (every variant reduces to alpha = |a| there).
template <int NV>
__device__ __forceinline__ void split_cell_gen(const double* Uc, int split, double alpha, double a_adv,
                                               double gamma, const CellPlanes<NV>& s, int si) {
    const double gm1 = gamma - 1.0;
    if (NV == 1 || split == 0) {
        split_cell<NV>(Uc, alpha, a_adv, gm1, s, si);
        return;
    }
    const double rho = Uc[0], mn = Uc[1], E = Uc[NV - 1];
    const double mt = NV == 4 ? Uc[2] : 0.0;
    const double rs = rsqrt(rho);
    const double rr = rs * rs;
    const double un = mn * rr;
    const double ut = mt * rr;
    const double kin = NV == 4 ? 0.5 * fma(mn, un, mt * ut) : 0.5 * (mn * un);
    const double p = gm1 * (E - kin);
    const double Ep = E + p;
    if (split == 3) {
        const double c = sqrt(gamma * p * rr);
        const double l1 = un - c, l3 = un + c;
        const double lp[3] = {0.5 * (l1 + fabs(l1)), 0.5 * (un + fabs(un)), 0.5 * (l3 + fabs(l3))};
        const double lm[3] = {0.5 * (l1 - fabs(l1)), 0.5 * (un - fabs(un)), 0.5 * (l3 - fabs(l3))};
        const double k0 = rho / (2.0 * gamma);
        const double q2 = NV == 4 ? fma(un, un, ut * ut) : un * un;
        const double vv = NV == 4 ? ut * ut : 0.0;
        const double e1 = 0.5 * fma(l1, l1, vv), e3 = 0.5 * fma(l3, l3, vv);     // ((u -+ c)^2 + v^2)/2
        const double w13 = (3.0 - gamma) * c * c / (2.0 * gm1);
        const double g2 = 2.0 * gm1;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const double* l = side == 0 ? lp : lm;
            double* h = side == 0 ? s.hp : s.hm;
            const double m0 = fma(g2, l[1], l[0] + l[2]);
            h[si] = k0 * m0;
            h[s.NC + si] = k0 * fma(g2 * l[1], un, fma(l[0], l1, l[2] * l3));
            if (NV == 4) h[2 * s.NC + si] = k0 * (m0 * ut);
            h[(NV - 1) * s.NC + si] = k0 * fma(gm1 * l[1], q2, fma(l[0], e1, fma(l[2], e3, (l[0] + l[2]) * w13)));
        }
    } else {
        const double hun = 0.5 * un;
        double hF[NV];
        hF[0] = 0.5 * mn;
        hF[1] = fma(mn, hun, 0.5 * p);
        if (NV == 4) hF[2] = mt * hun;
        hF[NV - 1] = hun * Ep;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            s.hp[k * s.NC + si] = hF[k];
            s.hm[k * s.NC + si] = 0.5 * Uc[k];
        }
        // local LF: the cell's |u_n| + c (the interface takes the largest of its six cells;
        // the per-field splitting reads global speeds instead)
        if (split == 2) s.sp[si] = fabs(un) + sqrt(gamma * p * rr);
    }
    s.sr[si] = rho * rs;
    s.un[si] = un;
    s.H[si] = Ep * rr;
    if (NV == 4) s.ut[si] = ut;
}

// Numerical flux F^ at the interface between the stencil's cells 2 and 3, the stencil being
// the six cells base + k*stride, k = 0..5 (cells i-2 .. i+3 around x_{i+1/2}); for the
// Euler systems the planes dh+ of cells 0..3 and dh- of cells 1..4 must be filled
// (cell_diffs).  Fh is in the sweep direction's frame.
template <int NV>
__device__ __forceinline__ void interface_flux(const CellPlanes<NV>& s, int base, int stride,
                                               double gm1, double eps4, double kappa, double* Fh) {
    const int NC = s.NC;
    if (NV == 1) {
        Fh[0] = zn_split_flux(s.hp[base], s.hp[base + stride], s.hp[base + 2 * stride],
                              s.hp[base + 3 * stride], s.hp[base + 4 * stride],
                              s.hm[base + stride], s.hm[base + 2 * stride], s.hm[base + 3 * stride],
                              s.hm[base + 4 * stride], s.hm[base + 5 * stride], eps4, kappa);
        return;
    }
    // Roe average between the stencil's cells 2 and 3
    const int cl = base + 2 * stride, cr = base + 3 * stride;
    const double srl = s.sr[cl], srr = s.sr[cr];
    const double rsum = rcp_nr(srl + srr);
    const double wl = srl * rsum, wr = srr * rsum;
    const double u = fma(wl, s.un[cl], wr * s.un[cr]);
    const double v = NV == 4 ? fma(wl, s.ut[cl], wr * s.ut[cr]) : 0.0;
    const double H = fma(wl, s.H[cl], wr * s.H[cr]);
    const double q2 = NV == 4 ? fma(u, u, v * v) : u * u;
    const double c2 = gm1 * fma(-0.5, q2, H);
    const double rc = rsqrt(c2);
    const double c = c2 * rc;
    const double hrc = 0.5 * rc;
    const double hq2 = 0.5 * q2;
    const double hb1 = (0.5 * gm1) * (rc * rc);        // b1 / 2, b1 = (gamma - 1) / c^2
    const double hb2 = hq2 * hb1;                      // b2 / 2, b2 = q^2 b1 / 2
    // Projection onto the left eigenvectors of the Roe state (rows, direction frame)
    //   l_{u-c} = ( (b2 + u/c)/2, -(b1 u + 1/c)/2, -b1 v/2, b1/2 )
    //   l_u     = ( 1 - b2, b1 u, b1 v, -b1 )
    //   l_shear = ( -v, 0, 1, 0 )                          (2D only)
    //   l_{u+c} = ( (b2 - u/c)/2, -(b1 u - 1/c)/2, -b1 v/2, b1/2 )
    // evaluated through their shared parts: with W = u h_1 + v h_2 - h_E,
    // Z = b2 h_0 - b1 W and B = (u h_0 - h_1)/(2c),
    //   l_u.h = h_0 - Z,  l_{u-+c}.h = Z/2 +- B,  l_shear.h = h_2 - v h_0.
    auto project = [&](const double* h, double* g) {
        const double h0 = h[0], h1 = h[1], hE = h[NV - 1];
        const double W = NV == 4 ? fma(u, h1, fma(v, h[2], -hE)) : fma(u, h1, -hE);
        const double Zh = fma(hb2, h0, -(hb1 * W));          // Z / 2
        const double Bi = fma(u, h0, -h1);                   // 2 c B
        g[0] = fma(hrc, Bi, Zh);
        g[1] = fma(-2.0, Zh, h0);
        if (NV == 4) g[2] = fma(-v, h0, h[2]);
        g[NV - 1] = fma(-hrc, Bi, Zh);
    };
    auto project_at = [&](const double* planes, int i, double* g) {
        double h[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) h[k] = planes[k * NC + i];
        project(h, g);
    };
    // Each field's reconstructions need only the first differences of its stencil and the
    // centre value: plus side (g+ at cells 0..4) D_s = l.dh+ at cells s - 1, centre l.h+_2;
    // minus side, the mirrored stencil of g- at cells 5..1, D_s = -l.dh- at cells 5 - s,
    // centre l.h-_3; both centres at once as l.(h+_2 + h-_3).
    double Dp[4][NV], Dm[4][NV], C[NV];
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        project_at(s.dp, base + st * stride, Dp[st]);
        project_at(s.dm, base + (st + 1) * stride, Dm[st]);
    }
    {
        double hc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) hc[k] = s.hp[k * NC + base + 2 * stride] + s.hm[k * NC + base + 3 * stride];
        project(hc, C);
    }
    double gh[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double fm = zn_flux_d(-Dm[3][k], -Dm[2][k], -Dm[1][k], -Dm[0][k], C[k], eps4, kappa);
        gh[k] = zn_flux_d(Dp[0][k], Dp[1][k], Dp[2][k], Dp[3][k], fm, eps4, kappa);
    }
    // back-projection F^ = R g^ with the right eigenvectors (columns)
    //   r_{u-c} = (1, u-c, [v,] H-uc), r_u = (1, u, [v,] q^2/2), r_shear = (0, 0, 1, v),
    //   r_{u+c} = (1, u+c, [v,] H+uc)
    const double uc = u * c;
    if (NV == 3) {
        const double d20 = gh[2] - gh[0];
        Fh[0] = gh[0] + gh[1] + gh[2];
        Fh[1] = fma(u, Fh[0], c * d20);
        Fh[2] = fma(H, gh[0] + gh[2], fma(uc, d20, hq2 * gh[1]));
    } else {
        const double d30 = gh[3] - gh[0];
        Fh[0] = gh[0] + gh[1] + gh[3];
        Fh[1] = fma(u, Fh[0], c * d30);
        Fh[2] = fma(v, Fh[0], gh[2]);
        Fh[3] = fma(H, gh[0] + gh[3], fma(uc, d30, fma(hq2, gh[1], v * gh[2])));
    }
}

// The interface flux of the generic kernels: weights and splitting chosen at run time.
// Splits 0 and 3 (DIFF) project the cell split fluxes h+- (their differences and centres);
// splits 1 and 2 project F/2 and U/2 of the six cells (their differences and centres) and
// split each field k with its speed alpha_k: g+- = l_k.(F/2) +- alpha_k l_k.(U/2),
// alpha_k = alpha_f[kind of field k] (split 1; kinds 0 u-c, 1 u, 2 u+c) or the largest
// |u_n| + c of the six cells (split 2).  The planes dh+- must be filled (cell_diffs).
template <int NV, bool DIFF>
__device__ __forceinline__ void interface_flux_gen(const CellPlanes<NV>& s, int base, int stride, double gm1,
                                                   double eps4, double kappa, int weights, int split,
                                                   const double* alpha_f, double* Fh) {
    const int NC = s.NC;
    if (NV == 1) {
        const double p0 = s.hp[base], p1 = s.hp[base + stride], p2 = s.hp[base + 2 * stride];
        const double p3 = s.hp[base + 3 * stride], p4 = s.hp[base + 4 * stride];
        const double m0 = s.hm[base + stride], m1 = s.hm[base + 2 * stride], m2 = s.hm[base + 3 * stride];
        const double m3 = s.hm[base + 4 * stride], m4 = s.hm[base + 5 * stride];
        Fh[0] = zn_flux_w(p0, p1, p2, p3, p4, eps4, kappa, weights) +
                zn_flux_w(m4, m3, m2, m1, m0, eps4, kappa, weights);
        return;
    }
    const int cl = base + 2 * stride, cr = base + 3 * stride;
    const double srl = s.sr[cl], srr = s.sr[cr];
    const double rsum = rcp_nr(srl + srr);
    const double wl = srl * rsum, wr = srr * rsum;
    const double u = fma(wl, s.un[cl], wr * s.un[cr]);
    const double v = NV == 4 ? fma(wl, s.ut[cl], wr * s.ut[cr]) : 0.0;
    const double H = fma(wl, s.H[cl], wr * s.H[cr]);
    const double q2 = NV == 4 ? fma(u, u, v * v) : u * u;
    const double c2 = gm1 * fma(-0.5, q2, H);
    const double rc = rsqrt(c2);
    const double c = c2 * rc;
    const double hrc = 0.5 * rc;
    const double hq2 = 0.5 * q2;
    const double hb1 = (0.5 * gm1) * (rc * rc);        // b1 / 2, b1 = (gamma - 1) / c^2
    const double hb2 = hq2 * hb1;                      // b2 / 2, b2 = q^2 b1 / 2
    // left eigenvectors through their shared parts, as in interface_flux
    auto project = [&](const double* h, double* g) {
        const double h0 = h[0], h1 = h[1], hE = h[NV - 1];
        const double W = NV == 4 ? fma(u, h1, fma(v, h[2], -hE)) : fma(u, h1, -hE);
        const double Zh = fma(hb2, h0, -(hb1 * W));          // Z / 2
        const double Bi = fma(u, h0, -h1);                   // 2 c B
        g[0] = fma(hrc, Bi, Zh);
        g[1] = fma(-2.0, Zh, h0);
        if (NV == 4) g[2] = fma(-v, h0, h[2]);
        g[NV - 1] = fma(-hrc, Bi, Zh);
    };
    auto project_at = [&](const double* planes, int i, double* g) {
        double h[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) h[k] = planes[k * NC + i];
        project(h, g);
    };
    double gh[NV];
    if (DIFF) {
        // splits 0 and 3, split fluxes per cell: the stencil differences and both centre
        // values projected as in interface_flux (the planes dh+- filled by cell_diffs)
        double Dp[4][NV], Dm[4][NV], C[NV];
#pragma unroll
        for (int st = 0; st < 4; ++st) {
            project_at(s.dp, base + st * stride, Dp[st]);
            project_at(s.dm, base + (st + 1) * stride, Dm[st]);
        }
        double hc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) hc[k] = s.hp[k * NC + base + 2 * stride] + s.hm[k * NC + base + 3 * stride];
        project(hc, C);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const double fm = zn_flux_w_d(-Dm[3][k], -Dm[2][k], -Dm[1][k], -Dm[0][k], C[k], eps4, kappa, weights);
            gh[k] = zn_flux_w_d(Dp[0][k], Dp[1][k], Dp[2][k], Dp[3][k], fm, eps4, kappa, weights);
        }
    } else {
        // splits 1 and 2: hp = F/2 and hm = U/2 per cell, each field split with its speed after
        // the projection, g+-_c = l.F_c/2 +- a_k l.U_c/2; differences g+-_c - g+-_{c+1} =
        // l.dF_c/2 +- a_k l.dU_c/2 (dh+- of cells 0..4), both centres at once as
        // l.(F_2 + F_3)/2 + a_k l.(U_2 - U_3)/2
        double ak[NV];
        if (split == 2) {
            double a = s.sp[base];
#pragma unroll
            for (int st = 1; st < 6; ++st) a = fmax(a, s.sp[base + st * stride]);
#pragma unroll
            for (int k = 0; k < NV; ++k) ak[k] = a;
        } else {
            ak[0] = alpha_f[0];
            ak[1] = alpha_f[1];
            if (NV == 4) ak[2] = alpha_f[1];
            ak[NV - 1] = alpha_f[2];
        }
        // plus side D_s = g+_{s-1} - g+_s (cells 0..3 of dh), minus side the mirrored
        // D_s = -(g-_{5-s} - g-_{6-s}) (cells 4..1), combined as each point is projected
        double Dp[4][NV], Dm[4][NV], cF[NV], cU[NV];
#pragma unroll
        for (int st = 0; st < 5; ++st) {
            double gF[NV], gU[NV];
            project_at(s.dp, base + st * stride, gF);
            project_at(s.dm, base + st * stride, gU);
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                if (st <= 3) Dp[st][k] = fma(ak[k], gU[k], gF[k]);
                if (st >= 1) Dm[st - 1][k] = fma(ak[k], gU[k], -gF[k]);
            }
        }
        {
            double hf[NV], hu[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                hf[k] = s.hp[k * NC + base + 2 * stride] + s.hp[k * NC + base + 3 * stride];
                hu[k] = s.hm[k * NC + base + 2 * stride] - s.hm[k * NC + base + 3 * stride];
            }
            project(hf, cF);
            project(hu, cU);
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const double C = fma(ak[k], cU[k], cF[k]);
            const double fm = zn_flux_w_d(Dm[3][k], Dm[2][k], Dm[1][k], Dm[0][k], C, eps4, kappa, weights);
            gh[k] = zn_flux_w_d(Dp[0][k], Dp[1][k], Dp[2][k], Dp[3][k], fm, eps4, kappa, weights);
        }
    }
    const double uc = u * c;
    if (NV == 3) {
        const double d20 = gh[2] - gh[0];
        Fh[0] = gh[0] + gh[1] + gh[2];
        Fh[1] = fma(u, Fh[0], c * d20);
        Fh[2] = fma(H, gh[0] + gh[2], fma(uc, d20, hq2 * gh[1]));
    } else {
        const double d30 = gh[3] - gh[0];
        Fh[0] = gh[0] + gh[1] + gh[3];
        Fh[1] = fma(u, Fh[0], c * d30);
        Fh[2] = fma(v, Fh[0], gh[2]);
        Fh[3] = fma(H, gh[0] + gh[3], fma(uc, d30, fma(hq2, gh[1], v * gh[2])));
    }
}

}  // namespace wz
