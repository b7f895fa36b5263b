// Interface-flux kernels: global Lax-Friedrichs splitting, Roe-averaged characteristic
// projection and WENO-ZN reconstruction of both split parts, one thread per interface.
// The generic instantiations (GEN = 1: splittings that project the cell split fluxes, global
// LF and Steger-Warming; GEN = 2: those that split per field after the projection, per-field
// and local LF) take the weight function and the flux splitting at run
// time (WENO-Z / linear / Jiang-Shu weights; per-field LF, local LF, Steger-Warming); the
// default scheme keeps its own instantiations.
//
// A block owns a tile of TI interfaces along the sweep direction times TA grid lines.  It
// first computes, once per cell of the tile plus its 3+2 halo cells, the split fluxes
// h+- = (F +- alpha U)/2 and the Roe-average ingredients (sqrt(rho), velocities, H) into
// shared memory; then every thread turns the six cells around its interface into
// F^_{i-1/2} = R (g^+ + g^-).  No interface is computed twice.
#include <atomic>

#include "euler_device.cuh"
#include "launch.h"

namespace wz {

namespace {

// Tile shapes: TI interfaces along the sweep x TA lines across it, THREADS per block.
// Long 1D lines use 507-interface tiles (512 cells with the halo: two full rounds of the cell
// and difference passes); short ones (fewer tiles than twice the SM count) use 64-interface
// tiles of 64 threads so that every SM gets work.
template <int NV, int DIR, bool SMALL = false> struct Tile;
template <> struct Tile<1, 0, false> { static constexpr int TI = 507, TA = 1, THREADS = 256; };
template <> struct Tile<3, 0, false> { static constexpr int TI = 507, TA = 1, THREADS = 256; };
template <> struct Tile<1, 0, true> { static constexpr int TI = 64, TA = 1, THREADS = 64; };
template <> struct Tile<3, 0, true> { static constexpr int TI = 64, TA = 1, THREADS = 64; };
template <> struct Tile<4, 0, false> { static constexpr int TI = 128, TA = 4, THREADS = 256; };
template <> struct Tile<4, 1, false> { static constexpr int TI = 32, TA = 16, THREADS = 256; };

// One tile of a sweep: tile ta along the sweep direction, tile tc across it.
template <int NV, int DIR, bool SMALL, int GEN>
__device__ __forceinline__ void flux_tile(const FluxArgs& a, int ta, int tc, double* smem) {
    constexpr int TI = Tile<NV, DIR, SMALL>::TI, TA = Tile<NV, DIR, SMALL>::TA;
    constexpr int kThreads = Tile<NV, DIR, SMALL>::THREADS;
    constexpr int CL = TI + 5;            // cells per line in the tile
    constexpr int NC = CL * TA;           // cells per tile
    const CellPlanes<NV> sp(smem, NC);

    const int n = DIR == 0 ? a.nx : a.ny;           // cells along the sweep
    const int nlines = DIR == 0 ? a.ny : a.nx;
    const int j0 = ta * TI;                         // first interface of the tile
    const int l0 = tc * TA;                         // first line of the tile
    const int64_t nc = int64_t(a.nx) * a.ny;
    // cells this tile's interfaces use along the sweep (the last tile of a line may hold
    // fewer than TI interfaces, e.g. only the boundary interface n)
    const int cl_used = min(TI, n + 1 - j0) + 5;

    // cell (line l, along index lc) -> shared index; the fastest thread index runs along
    // the contiguous direction of global memory
    auto sidx = [](int l, int lc) { return DIR == 0 ? l * CL + lc : lc * TA + l; };
    constexpr int kStride = DIR == 0 ? 1 : TA;      // shared-index step along the sweep

    const double alpha = NV == 1 ? fabs(a.adv_speed) : __longlong_as_double((long long)a.alpha_bits[DIR]);
    const double gm1 = a.gamma - 1.0;
    double alpha_f[3] = {0.0, 0.0, 0.0};           // per-field speeds of this direction
    if (GEN == 2 && NV > 1 && a.split == 1)
        for (int k = 0; k < 3; ++k) alpha_f[k] = __longlong_as_double((long long)a.alpha_f_bits[DIR * 3 + k]);

    // ---- per-cell quantities -------------------------------------------------------
    for (int idx = threadIdx.x; idx < NC; idx += kThreads) {
        const int l = DIR == 0 ? idx / CL : idx % TA;
        const int lc = DIR == 0 ? idx % CL : idx / TA;
        if (lc >= cl_used) continue;
        const int line = min(l0 + l, nlines - 1);
        const int gi = j0 - 3 + lc;
        const int g = ghost_src(gi, n, a.bc);
        const int64_t cell = DIR == 0 ? int64_t(line) * a.nx + g : int64_t(g) * a.nx + line;
        // direction frame: (rho, m_n, m_t, E)
        double Uc[NV];
        Uc[0] = a.U[cell];
        if (NV > 1) {
            Uc[1] = a.U[(DIR == 0 ? 1 : 2) * nc + cell];
            if (NV == 4) Uc[2] = a.U[(DIR == 0 ? 2 : 1) * nc + cell];
            Uc[NV - 1] = a.U[(NV - 1) * nc + cell];
            if (a.bc == 2 && ghost_mirrored(gi, n, a.bc)) Uc[1] = -Uc[1];   // wall mirror image
        }
        if (GEN != 0) split_cell_gen<NV>(Uc, a.split, alpha, a.adv_speed, a.gamma, sp, sidx(l, lc));
        else split_cell<NV>(Uc, alpha, a.adv_speed, gm1, sp, sidx(l, lc));
    }
    __syncthreads();
    if (NV > 1) {
        // the split-flux differences of neighbouring cells along the sweep
        for (int idx = threadIdx.x; idx < NC; idx += kThreads) {
            const int l = DIR == 0 ? idx / CL : idx % TA;
            const int lc = DIR == 0 ? idx % CL : idx / TA;
            if (lc < cl_used - 1) cell_diffs<NV>(sp, sidx(l, lc), kStride);
        }
        __syncthreads();
    }

    // ---- interfaces ----------------------------------------------------------------
    const int nint = DIR == 0 ? a.nx + 1 : a.ny + 1;
    for (int idx = threadIdx.x; idx < TI * TA; idx += kThreads) {
        const int l = DIR == 0 ? idx / TI : idx % TA;
        const int jl = DIR == 0 ? idx % TI : idx / TA;
        const int j = j0 + jl, line = l0 + l;
        if (j >= nint || line >= nlines) continue;
        double Fh[NV];
        if (GEN != 0)
            interface_flux_gen<NV, GEN == 1>(sp, sidx(l, jl), kStride, gm1, a.eps4, a.kappa, a.weights,
                                             a.split, alpha_f, Fh);
        else
            interface_flux<NV>(sp, sidx(l, jl), kStride, gm1, a.eps4, a.kappa, Fh);
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

template <int NV, int DIR, bool SMALL, int GEN>
__global__ void __launch_bounds__(Tile<NV, DIR, SMALL>::THREADS, 2) flux_kernel(FluxArgs a) {
    extern __shared__ double smem[];
    pdl_wait();
    flux_tile<NV, DIR, SMALL, GEN>(a, DIR == 0 ? blockIdx.x : blockIdx.y, DIR == 0 ? blockIdx.y : blockIdx.x, smem);
}

// Both sweeps of a 2D stage in one grid, so that they share one tail: blocks [0, nbx) take
// the x tiles (along the sweep fastest, as flux_kernel<4, 0>), the others the y tiles
// (across the sweep fastest, as flux_kernel<4, 1>).
template <int GEN>
__global__ void __launch_bounds__(256, 2) flux_xy_kernel(FluxArgs ax, FluxArgs ay, int x_along, int nbx, int y_across) {
    static_assert(Tile<4, 0>::THREADS == 256 && Tile<4, 1>::THREADS == 256, "one block size for both sweeps");
    extern __shared__ double smem[];
    pdl_wait();
    const int b = int(blockIdx.x);
    if (b < nbx) {
        flux_tile<4, 0, false, GEN>(ax, b % x_along, b / x_along, smem);
    } else {
        const int q = b - nbx;
        flux_tile<4, 1, false, GEN>(ay, q / y_across, q % y_across, smem);
    }
}

template <int NV, int DIR, bool SMALL, int GEN>
constexpr size_t tile_smem() {
    return size_t((Tile<NV, DIR, SMALL>::TI + 5) * Tile<NV, DIR, SMALL>::TA) *
           (GEN != 0 ? CellPlanes<NV>::kPerCellGeneric : CellPlanes<NV>::kPerCellDefault) * sizeof(double);
}

template <int GEN>
cudaError_t launch_xy(const FluxArgs& ax, const FluxArgs& ay, cudaStream_t s) {
    constexpr size_t sx = tile_smem<4, 0, false, GEN>(), sy = tile_smem<4, 1, false, GEN>();
    constexpr size_t smem = sx > sy ? sx : sy;
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(flux_xy_kernel<GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    const int x_along = (ax.nx + 1 + Tile<4, 0>::TI - 1) / Tile<4, 0>::TI;
    const int nbx = x_along * ((ax.ny + Tile<4, 0>::TA - 1) / Tile<4, 0>::TA);
    const int y_across = (ay.nx + Tile<4, 1>::TA - 1) / Tile<4, 1>::TA;
    const int nby = y_across * ((ay.ny + 1 + Tile<4, 1>::TI - 1) / Tile<4, 1>::TI);
    return launch_pdl(flux_xy_kernel<GEN>, dim3(unsigned(nbx + nby)), dim3(256), smem, s, ax, ay, x_along, nbx,
                      y_across);
}

template <int NV, int DIR, bool SMALL, int GEN>
cudaError_t launch_one(const FluxArgs& a, cudaStream_t s) {
    constexpr int TI = Tile<NV, DIR, SMALL>::TI, TA = Tile<NV, DIR, SMALL>::TA;
    constexpr size_t smem = tile_smem<NV, DIR, SMALL, GEN>();
    // the dynamic shared-memory limit is a per-device function attribute
    static std::atomic<unsigned long long> configured{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(configured.load() & bit)) {
        e = cudaFuncSetAttribute(flux_kernel<NV, DIR, SMALL, GEN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem));
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    const int n = DIR == 0 ? a.nx : a.ny;
    const int nlines = DIR == 0 ? a.ny : a.nx;
    const unsigned along = unsigned((n + 1 + TI - 1) / TI);
    const unsigned across = unsigned((nlines + TA - 1) / TA);
    dim3 grid = DIR == 0 ? dim3(along, across) : dim3(across, along);
    return launch_pdl(flux_kernel<NV, DIR, SMALL, GEN>, grid, dim3(Tile<NV, DIR, SMALL>::THREADS), smem, s, a);
}

int sm_count_cached() {
    static int sms = 0;
    if (sms > 0) return sms;
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
        sms = v;
    return sms > 0 ? sms : 152;
}

template <int GEN>
cudaError_t launch_flux_t(int system, int dir, const FluxArgs& a, cudaStream_t s) {
    if (system != 2) {
        // 1D: short lines take the small tiles so that every SM has work
        const int64_t big_tiles = (int64_t(a.nx) + Tile<3, 0>::TI) / Tile<3, 0>::TI * a.ny;
        const bool small = big_tiles < 2 * sm_count_cached();
        if (system == 0) return small ? launch_one<1, 0, true, GEN>(a, s) : launch_one<1, 0, false, GEN>(a, s);
        return small ? launch_one<3, 0, true, GEN>(a, s) : launch_one<3, 0, false, GEN>(a, s);
    }
    return dir == 0 ? launch_one<4, 0, false, GEN>(a, s) : launch_one<4, 1, false, GEN>(a, s);
}

}  // namespace

cudaError_t launch_flux_xy(const FluxArgs& ax, const FluxArgs& ay, cudaStream_t s) {
    if (ax.weights == 0 && ax.split == 0) return launch_xy<0>(ax, ay, s);
    const bool diff = ax.split == 0 || ax.split == 3;
    return diff ? launch_xy<1>(ax, ay, s) : launch_xy<2>(ax, ay, s);
}

cudaError_t launch_flux(int system, int dir, const FluxArgs& a, cudaStream_t s) {
    if (a.weights == 0 && (system == 0 || a.split == 0)) return launch_flux_t<0>(system, dir, a, s);
    // advection ignores the splitting
    const bool diff = system == 0 || a.split == 0 || a.split == 3;
    return diff ? launch_flux_t<1>(system, dir, a, s) : launch_flux_t<2>(system, dir, a, s);
}

}  // namespace wz
