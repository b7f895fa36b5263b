// Interface-flux kernels: global Lax-Friedrichs splitting, Roe-averaged characteristic
// projection and WENO-ZN reconstruction of both split parts, one thread per interface.
//
// A block owns a tile of TI interfaces along the sweep direction times TA grid lines.  It
// first computes, once per cell of the tile plus its 3+2 halo cells, the split fluxes
// h+- = (F +- alpha U)/2 and the Roe-average ingredients (sqrt(rho), velocities, H) into
// shared memory; then every thread turns the six cells around its interface into
// F^_{i-1/2} = R (g^+ + g^-).  No interface is computed twice.
#include <atomic>

#include "launch.h"

namespace wz {

namespace {

constexpr int kThreads = 256;

// Tile shapes (interfaces along the sweep x lines across it).
template <int NV, int DIR> struct Tile;
template <> struct Tile<1, 0> { static constexpr int TI = 512, TA = 1; };
template <> struct Tile<3, 0> { static constexpr int TI = 512, TA = 1; };
template <> struct Tile<4, 0> { static constexpr int TI = 128, TA = 4; };
template <> struct Tile<4, 1> { static constexpr int TI = 32, TA = 16; };

template <int NV> struct SmemLayout {
    // number of doubles per cell in shared memory
    static constexpr int kPerCell = NV == 1 ? 2 : 2 * NV + (NV == 4 ? 4 : 3);
};

template <int NV, int DIR>
__global__ void __launch_bounds__(kThreads, 2) flux_kernel(FluxArgs a) {
    constexpr int TI = Tile<NV, DIR>::TI, TA = Tile<NV, DIR>::TA;
    constexpr int CL = TI + 5;            // cells per line in the tile
    constexpr int NC = CL * TA;           // cells per tile
    extern __shared__ double smem[];
    double* sHp = smem;                   // [NV][NC]
    double* sHm = sHp + NV * NC;          // [NV][NC]
    double* sSr = sHm + NV * NC;          // [NC]  sqrt(rho)
    double* sUn = sSr + NC;               // [NC]  normal velocity
    double* sH = sUn + NC;                // [NC]  total enthalpy
    double* sUt = sH + NC;                // [NC]  tangential velocity (NV == 4)

    const int n = DIR == 0 ? a.nx : a.ny;           // cells along the sweep
    const int nlines = DIR == 0 ? a.ny : a.nx;
    const int j0 = (DIR == 0 ? blockIdx.x : blockIdx.y) * TI;   // first interface of the tile
    const int l0 = (DIR == 0 ? blockIdx.y : blockIdx.x) * TA;   // first line of the tile
    const int64_t nc = int64_t(a.nx) * a.ny;

    // cell (line l, along index lc) -> shared index; the fastest thread index runs along
    // the contiguous direction of global memory
    auto sidx = [](int l, int lc) { return DIR == 0 ? l * CL + lc : lc * TA + l; };

    double alpha, half_a;
    if (NV == 1) alpha = fabs(a.adv_speed);
    else alpha = __longlong_as_double((long long)a.alpha_bits[DIR]);
    half_a = 0.5 * alpha;
    const double gm1 = a.gamma - 1.0;

    // ---- per-cell quantities -------------------------------------------------------
    for (int idx = threadIdx.x; idx < NC; idx += kThreads) {
        const int l = DIR == 0 ? idx / CL : idx % TA;
        const int lc = DIR == 0 ? idx % CL : idx / TA;
        const int line = min(l0 + l, nlines - 1);
        const int g = ghost_src(j0 - 3 + lc, n, a.bc);
        const int64_t cell = DIR == 0 ? int64_t(line) * a.nx + g : int64_t(g) * a.nx + line;
        const int si = sidx(l, lc);
        if (NV == 1) {
            const double u = a.U[cell];
            const double f = a.adv_speed * u;
            sHp[si] = 0.5 * fma(alpha, u, f);
            sHm[si] = 0.5 * fma(-alpha, u, f);
            continue;
        }
        // direction frame: (rho, m_n, m_t, E)
        const double rho = a.U[cell];
        const double mn = a.U[(DIR == 0 ? 1 : 2) * nc + cell];
        const double mt = NV == 4 ? a.U[(DIR == 0 ? 2 : 1) * nc + cell] : 0.0;
        const double E = a.U[(NV - 1) * nc + cell];
        const double rs = rsqrt(rho);
        const double rr = rs * rs;                         // 1 / rho
        const double un = mn * rr;
        const double ut = mt * rr;
        const double kin = NV == 4 ? 0.5 * fma(mn, un, mt * ut) : 0.5 * (mn * un);
        const double p = gm1 * (E - kin);
        const double Ep = E + p;
        // half the physical flux, F/2 = (m_n, m_n u_n + p, m_t u_n, u_n (E + p)) / 2
        const double hun = 0.5 * un;
        double hF[NV], Uc[NV];
        Uc[0] = rho; Uc[1] = mn; Uc[NV - 1] = E;
        hF[0] = 0.5 * mn;
        hF[1] = fma(mn, hun, 0.5 * p);
        if (NV == 4) { Uc[2] = mt; hF[2] = mt * hun; }
        hF[NV - 1] = hun * Ep;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            sHp[k * NC + si] = fma(half_a, Uc[k], hF[k]);
            sHm[k * NC + si] = fma(-half_a, Uc[k], hF[k]);
        }
        sSr[si] = rho * rs;                                // sqrt(rho)
        sUn[si] = un;
        sH[si] = Ep * rr;
        if (NV == 4) sUt[si] = ut;
    }
    __syncthreads();

    // ---- interfaces ----------------------------------------------------------------
    const int nint = DIR == 0 ? a.nx + 1 : a.ny + 1;
    for (int idx = threadIdx.x; idx < TI * TA; idx += kThreads) {
        const int l = DIR == 0 ? idx / TI : idx % TA;
        const int jl = DIR == 0 ? idx % TI : idx / TA;
        const int j = j0 + jl, line = l0 + l;
        if (j >= nint || line >= nlines) continue;
        double Fh[NV];
        if (NV == 1) {
            Fh[0] = zn_split_flux(sHp[sidx(l, jl)], sHp[sidx(l, jl + 1)], sHp[sidx(l, jl + 2)],
                                  sHp[sidx(l, jl + 3)], sHp[sidx(l, jl + 4)],
                                  sHm[sidx(l, jl + 1)], sHm[sidx(l, jl + 2)], sHm[sidx(l, jl + 3)],
                                  sHm[sidx(l, jl + 4)], sHm[sidx(l, jl + 5)], a.eps4, a.A4, a.fast_rcp != 0);
        } else {
            // Roe average between cells j-1 and j (local jl+2, jl+3)
            const int cl = sidx(l, jl + 2), cr = sidx(l, jl + 3);
            const double srl = sSr[cl], srr = sSr[cr];
            const double rsum = rcp_nr(srl + srr);
            const double wl = srl * rsum, wr = srr * rsum;
            const double u = fma(wl, sUn[cl], wr * sUn[cr]);
            const double v = NV == 4 ? fma(wl, sUt[cl], wr * sUt[cr]) : 0.0;
            const double H = fma(wl, sH[cl], wr * sH[cr]);
            const double q2 = NV == 4 ? fma(u, u, v * v) : u * u;
            const double c2 = gm1 * fma(-0.5, q2, H);
            const double rc = rsqrt(c2);
            const double c = c2 * rc;
            const double b1 = gm1 * (rc * rc);             // (gamma - 1) / c^2
            const double b2 = 0.5 * q2 * b1;
            const double hrc = 0.5 * rc;
            // Projection onto the left eigenvectors of the Roe state (rows, direction frame)
            //   l_{u-c} = ( (b2 + u/c)/2, -(b1 u + 1/c)/2, -b1 v/2, b1/2 )
            //   l_u     = ( 1 - b2, b1 u, b1 v, -b1 )
            //   l_shear = ( -v, 0, 1, 0 )                          (2D only)
            //   l_{u+c} = ( (b2 - u/c)/2, -(b1 u - 1/c)/2, -b1 v/2, b1/2 )
            // evaluated through their shared parts: with W = u h_1 + v h_2 - h_E,
            // Z = b2 h_0 - b1 W and B = (u h_0 - h_1)/(2c),
            //   l_u.h = h_0 - Z,  l_{u-+c}.h = Z/2 +- B,  l_shear.h = h_2 - v h_0.
            auto project = [&](const double* hs, int i, double* g) {
                const double h0 = hs[i], h1 = hs[NC + i], hE = hs[(NV - 1) * NC + i];
                const double W = NV == 4 ? fma(u, h1, fma(v, hs[2 * NC + i], -hE)) : fma(u, h1, -hE);
                const double Z = fma(b2, h0, -(b1 * W));
                const double B = hrc * fma(u, h0, -h1);
                g[0] = fma(0.5, Z, B);
                g[1] = h0 - Z;
                if (NV == 4) g[2] = fma(-v, h0, hs[2 * NC + i]);
                g[NV - 1] = fma(0.5, Z, -B);
            };
            double gp[5][NV], gm[5][NV];
#pragma unroll
            for (int st = 0; st < 5; ++st) {
                project(sHp, sidx(l, jl + st), gp[st]);
                project(sHm, sidx(l, jl + 1 + st), gm[st]);
            }
            double gh[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k)
                gh[k] = zn_split_flux(gp[0][k], gp[1][k], gp[2][k], gp[3][k], gp[4][k],
                                      gm[0][k], gm[1][k], gm[2][k], gm[3][k], gm[4][k], a.eps4, a.A4,
                                      a.fast_rcp != 0);
            // back-projection F^ = R g^ with the right eigenvectors (columns)
            const double uc = u * c;
            if (NV == 3) {
                const double d20 = gh[2] - gh[0];
                Fh[0] = gh[0] + gh[1] + gh[2];
                Fh[1] = fma(u, Fh[0], c * d20);
                Fh[2] = fma(H, gh[0] + gh[2], fma(uc, d20, 0.5 * q2 * gh[1]));
            } else {
                const double d30 = gh[3] - gh[0];
                Fh[0] = gh[0] + gh[1] + gh[3];
                Fh[1] = fma(u, Fh[0], c * d30);
                Fh[2] = fma(v, Fh[0], gh[2]);
                Fh[3] = fma(H, gh[0] + gh[3], fma(uc, d30, fma(0.5 * q2, gh[1], v * gh[2])));
            }
        }
        // store, undoing the direction frame
        if (DIR == 0) {
            const int64_t base = int64_t(line) * (a.nx + 1) + j;
            const int64_t stride = int64_t(a.ny) * (a.nx + 1);
#pragma unroll
            for (int k = 0; k < NV; ++k) a.Fout[k * stride + base] = Fh[k];
        } else {
            const int64_t base = int64_t(j) * a.nx + line;
            const int64_t stride = int64_t(a.ny + 1) * a.nx;
            a.Fout[base] = Fh[0];
            a.Fout[2 * stride + base] = Fh[1];    // y-momentum flux
            a.Fout[1 * stride + base] = Fh[2];    // x-momentum flux
            a.Fout[3 * stride + base] = Fh[3];
        }
    }
}

template <int NV, int DIR>
cudaError_t launch_one(const FluxArgs& a, cudaStream_t s) {
    constexpr int TI = Tile<NV, DIR>::TI, TA = Tile<NV, DIR>::TA;
    constexpr int NC = (TI + 5) * TA;
    constexpr size_t smem = size_t(NC) * SmemLayout<NV>::kPerCell * sizeof(double);
    // the dynamic shared-memory limit is a per-device function attribute
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(flux_kernel<NV, DIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem));
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    const int n = DIR == 0 ? a.nx : a.ny;
    const int nlines = DIR == 0 ? a.ny : a.nx;
    const unsigned along = unsigned((n + 1 + TI - 1) / TI);
    const unsigned across = unsigned((nlines + TA - 1) / TA);
    dim3 grid = DIR == 0 ? dim3(along, across) : dim3(across, along);
    flux_kernel<NV, DIR><<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_flux(int system, int dir, const FluxArgs& a, cudaStream_t s) {
    if (system == 0) return launch_one<1, 0>(a, s);
    if (system == 1) return launch_one<3, 0>(a, s);
    return dir == 0 ? launch_one<4, 0>(a, s) : launch_one<4, 1>(a, s);
}

}  // namespace wz
