// Batched 1D Euler: many independent problems of uneven size advanced together, one
// persistent launch per SSP-RK3 stage.
//
// Layout: the instances' conserved variables are concatenated per variable,
// U[3][total], instance b occupying columns off[b] .. off[b+1]-1.  Each instance is split
// into tiles of TI-1 cells (TI interfaces); tile_off[b] is the prefix count of tiles, so
// the flat work list is implicit and a block finds its instance by binary search.  A tile
// computes the split fluxes of its TI+5 cells, the TI interface fluxes, the flux
// difference and the stage update of its cells, and folds the LF speed of the updated
// cells into the instance's slot for the next stage (bit-pattern atomicMax).
//
// Per-instance state (device arrays in the workspace): LF speeds alpha[3][B] (one slot per
// RK stage, rotated statically: stage s reads slot s, accumulates slot s+1 mod 3 and
// clears slot s+2 mod 3), the step dt[B] of the current RK3 step (CFL, from U^n) and the
// time t[B].  Instances that reached t_final take dt = 0 and are skipped.
#include "euler_device.cuh"
#include "launch.h"
#include "speed_screen.cuh"

namespace wz {

namespace {

__device__ __forceinline__ double bits2d(unsigned long long b) { return __longlong_as_double((long long)b); }

template <int TI, int THREADS>
__global__ void __launch_bounds__(THREADS, 2) batch_stage_kernel(BatchArgs a) {
    constexpr int NV = 3;
    constexpr int CL = TI + 5;
    extern __shared__ double smem[];
    const CellPlanes<NV> sp(smem, CL);
    double* sF = smem + CL * CellPlanes<NV>::kPerCellDefault;  // [3][TI]
    __shared__ int s_inst;
    __shared__ float s_est[TI];                                // screened speed estimates
    __shared__ float s_red[THREADS / 32];

    const int ntiles = a.tile_off[a.B];
    const double gm1 = a.gamma - 1.0;
    const float gg1 = __double2float_rn(a.gamma * gm1);
    // the last state this thread evaluated exactly and its speed: a bit-identical state
    // (constant regions) reuses it
    double cs[NV];
    double csx = 0.0;
    bool cached = false;
    const int slot = a.stage, next = (a.stage + 1) % 3, clear = (a.stage + 2) % 3;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = a.B;                               // tile_off[lo] <= tile < tile_off[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (a.tile_off[mid] <= tile) lo = mid;
                else hi = mid;
            }
            s_inst = lo;
        }
        __syncthreads();
        const int b = s_inst;
        const int64_t o = a.off[b];
        const int n = int(a.off[b + 1] - o);
        const int c0 = (tile - a.tile_off[b]) * (TI - 1);
        const int ncell = min(TI - 1, n - c0);
        const bool first = tile == a.tile_off[b];
        const double dxb = a.dx[b];

        // step of this RK3 step: CFL from U^n (stage 0), in the oracle's operation order
        double dt;
        if (a.stage == 0) {
            const double ax = bits2d(a.alpha[slot * a.B + b]);
            dt = __ddiv_rn(__dmul_rn(a.cfl, dxb), ax);
            if (a.t_final > 0.0) {
                const double rem = a.t_final - a.t[b];
                dt = rem > 0.0 ? (dt > rem ? rem : dt) : 0.0;
            }
            if (first && threadIdx.x == 0) a.dt[b] = dt;
        } else {
            dt = a.dt[b];
        }
        if (first && threadIdx.x == 0) {
            a.alpha[clear * a.B + b] = 0ull;
            if (a.stage == 2) a.t[b] += dt;
        }
        if (dt == 0.0) {                    // finished instance: the state stays as it is
            if (a.stage < 2)
                for (int c = threadIdx.x; c < ncell; c += THREADS)
#pragma unroll
                    for (int k = 0; k < NV; ++k) a.out[k * a.total + o + c0 + c] = a.Us[k * a.total + o + c0 + c];
            __syncthreads();
            continue;
        }
        const double alpha = bits2d(a.alpha[slot * a.B + b]);

        // the cells interfaces c0 .. c0 + ncell use (an instance's last tile may hold fewer)
        const int cl_used = ncell + 6;
        for (int i = threadIdx.x; i < cl_used; i += THREADS) {
            const int g = ghost_src(c0 - 3 + i, n, a.bc);
            double Uc[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) Uc[k] = a.Us[k * a.total + o + g];
            split_cell<NV>(Uc, alpha, 0.0, gm1, sp, i);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cl_used - 1; i += THREADS) cell_diffs<NV>(sp, i, 1);
        __syncthreads();
        for (int jl = threadIdx.x; jl <= ncell; jl += THREADS) {     // interfaces c0 .. c0+ncell
            double Fh[NV];
            interface_flux<NV>(sp, jl, 1, gm1, a.eps4, a.kappa, Fh);
#pragma unroll
            for (int k = 0; k < NV; ++k) sF[k * TI + jl] = Fh[k];
        }
        __syncthreads();
        // the stage as base - kx dF with the RK weight and dt/dx folded into kx (Eq. (2))
        const double kx = (a.stage == 0 ? 1.0 : (a.stage == 1 ? 0.25 : 2.0 / 3.0)) * dt / dxb;
        double mx = 0.0, unused = 0.0;
        bool bad = false;
        float emax = 0.0f;
        for (int c = threadIdx.x; c < ncell; c += THREADS) {
            const int64_t gc = o + c0 + c;
            double r[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const double dF = sF[k * TI + c + 1] - sF[k * TI + c];
                const double us = a.Us[k * a.total + gc];
                double base = us;
                if (a.stage == 1) base = fma(0.75, a.Un[k * a.total + gc], 0.25 * us);
                else if (a.stage == 2) base = fma(1.0 / 3.0, a.Un[k * a.total + gc], (2.0 / 3.0) * us);
                r[k] = fma(-kx, dF, base);
                a.out[k * a.total + gc] = r[k];
            }
            // the next stage's LF speed: estimate every cell, evaluate exactly only the cells
            // the tile-wide screen cannot rule out (-1 marks a cell without a bound)
            const SpeedEstimate est = estimate_speeds<NV>(r, gg1);
            s_est[c] = est.ok ? est.sx : -1.0f;
            emax = fmaxf(emax, est.sx);
        }
        emax = warp_max_f(emax);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = emax;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < THREADS / 32; ++w) emax = fmaxf(emax, s_red[w]);
        for (int c = threadIdx.x; c < ncell; c += THREADS) {
            const float e = s_est[c];
            if (e >= 0.0f && e < emax * kScreenKeep) continue;
            const int64_t gc = o + c0 + c;
            double r[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) r[k] = a.out[k * a.total + gc];      // this thread's own writes
            bool same = cached;
#pragma unroll
            for (int k = 0; k < NV; ++k) same = same && __double_as_longlong(r[k]) == __double_as_longlong(cs[k]);
            if (!same) {
                double sy;
                bad |= !wave_speeds<NV>(r, a.gamma, csx, sy);
#pragma unroll
                for (int k = 0; k < NV; ++k) cs[k] = r[k];
                cached = true;
            }
            mx = fmax(mx, csx);
        }
        if (bad) atomicOr(a.status, kStatusNonFinite);
        block_max2_atomic(mx, unused, &a.alpha[next * a.B + b], true);
        __syncthreads();
    }
}

// Per-instance LF speed of U into slot 0 (one block per instance), other slots, dt and t
// cleared.
__global__ void __launch_bounds__(256) batch_init_kernel(BatchArgs a) {
    const int b = blockIdx.x;
    const int64_t o = a.off[b];
    const int n = int(a.off[b + 1] - o);
    double mx = 0.0, unused = 0.0;
    bool bad = false;
    for (int c = threadIdx.x; c < n; c += 256) {
        double s[3] = {a.Us[o + c], a.Us[a.total + o + c], a.Us[2 * a.total + o + c]};
        double sx, sy;
        bad |= !wave_speeds<3>(s, a.gamma, sx, sy);
        mx = fmax(mx, sx);
    }
    if (bad) atomicOr(a.status, kStatusNonFinite);
    if (threadIdx.x == 0) {
        a.alpha[b] = 0ull;
        a.alpha[a.B + b] = 0ull;
        a.alpha[2 * a.B + b] = 0ull;
        a.dt[b] = 0.0;
        a.t[b] = 0.0;
    }
    __syncthreads();
    block_max2_atomic(mx, unused, &a.alpha[b], true);
}

template <int TI, int THREADS>
cudaError_t launch_stage(const BatchArgs& a, int grid, cudaStream_t s) {
    constexpr size_t smem = (size_t(TI + 5) * CellPlanes<3>::kPerCellDefault + 3 * TI) * sizeof(double);
    batch_stage_kernel<TI, THREADS><<<grid, THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int TI, int THREADS>
cudaError_t configure_one() {
    constexpr size_t smem = (size_t(TI + 5) * CellPlanes<3>::kPerCellDefault + 3 * TI) * sizeof(double);
    return cudaFuncSetAttribute(batch_stage_kernel<TI, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(smem));
}

template <int TI, int THREADS>
int resident_blocks() {
    // resident blocks per SM of this shape (same on every GB300; looked up once)
    static int cached = 0;
    if (cached > 0) return cached;
    constexpr size_t smem = (size_t(TI + 5) * CellPlanes<3>::kPerCellDefault + 3 * TI) * sizeof(double);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_stage_kernel<TI, THREADS>, THREADS, smem) !=
        cudaSuccess)
        return 1;
    cached = nb > 0 ? nb : 1;
    return cached;
}

}  // namespace

// The tile/thread shapes the batched kernel is compiled for (the autotuner's candidates).
const BatchShape kBatchShapes[kNumBatchShapes] = {{128, 128}, {256, 128}, {256, 256}, {512, 256}, {1024, 256}};

cudaError_t batch_configure() {
    cudaError_t e = configure_one<128, 128>();
    if (e == cudaSuccess) e = configure_one<256, 128>();
    if (e == cudaSuccess) e = configure_one<256, 256>();
    if (e == cudaSuccess) e = configure_one<512, 256>();
    if (e == cudaSuccess) e = configure_one<1024, 256>();
    // look the occupancies up now, outside any stream capture
    resident_blocks<128, 128>();
    resident_blocks<256, 128>();
    resident_blocks<256, 256>();
    resident_blocks<512, 256>();
    resident_blocks<1024, 256>();
    return e;
}

cudaError_t launch_batch_init(const BatchArgs& a, cudaStream_t s) {
    batch_init_kernel<<<a.B, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_batch_stage(int shape, const BatchArgs& a, int sms, cudaStream_t s) {
    switch (shape) {
        case 0: return launch_stage<128, 128>(a, sms * resident_blocks<128, 128>(), s);
        case 1: return launch_stage<256, 128>(a, sms * resident_blocks<256, 128>(), s);
        case 2: return launch_stage<256, 256>(a, sms * resident_blocks<256, 256>(), s);
        case 3: return launch_stage<512, 256>(a, sms * resident_blocks<512, 256>(), s);
        case 4: return launch_stage<1024, 256>(a, sms * resident_blocks<1024, 256>(), s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace wz
