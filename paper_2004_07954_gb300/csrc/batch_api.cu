// C ABI of the batched 1D Euler path (declarations and contracts in include/wenozn.h).
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "../../include/wenozn.h"
#include "launch.h"

using namespace wz;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct BatchLayout {
    size_t ctrl, off, tile_off, dx, alpha, dt, t, u1, u2, total;
};

BatchLayout batch_layout(int B, int64_t cells) {
    BatchLayout L;
    L.ctrl = 0;
    L.off = align_up(sizeof(Ctrl));
    L.tile_off = L.off + align_up(size_t(B + 1) * sizeof(int64_t));
    L.dx = L.tile_off + align_up(size_t(kNumBatchShapes) * (B + 1) * sizeof(int32_t));
    L.alpha = L.dx + align_up(size_t(B) * sizeof(double));
    L.dt = L.alpha + align_up(size_t(3) * B * sizeof(unsigned long long));
    L.t = L.dt + align_up(size_t(B) * sizeof(double));
    L.u1 = L.t + align_up(size_t(B) * sizeof(double));
    L.u2 = L.u1 + align_up(size_t(3) * cells * sizeof(double));
    L.total = L.u2 + align_up(size_t(3) * cells * sizeof(double));
    return L;
}

// Validates the parameters and the host offsets; returns the total cell count in *cells.
wenozn_status check_batch(const wenozn_batch_params* bp, const int64_t* offsets, int64_t* cells) {
    if (!bp || !offsets || !cells) return WENOZN_EINVAL;
    if (bp->nbatch < 1 || bp->nbatch > (1 << 24) || bp->flags != 0) return WENOZN_EINVAL;
    if (bp->bc != WENOZN_BC_PERIODIC && bp->bc != WENOZN_BC_OUTFLOW) return WENOZN_EINVAL;
    if (bp->shape < -1 || bp->shape >= kNumBatchShapes) return WENOZN_EINVAL;
    if (!(std::isfinite(bp->gamma) && bp->gamma > 1.0) || !(std::isfinite(bp->eps) && bp->eps > 0.0) ||
        !(std::isfinite(bp->A) && bp->A > 0.0) || !(std::isfinite(bp->cfl) && bp->cfl > 0.0) ||
        std::isnan(bp->t_final) || !zn_constants_ok(bp->eps, bp->A))
        return WENOZN_EINVAL;
    if (offsets[0] != 0) return WENOZN_EINVAL;
    for (int b = 0; b < bp->nbatch; ++b) {
        const int64_t n = offsets[b + 1] - offsets[b];
        if (n < 1 || n > (int64_t(1) << 30)) return WENOZN_EINVAL;
    }
    *cells = offsets[bp->nbatch];
    if (*cells > (int64_t(1) << 34)) return WENOZN_EINVAL;
    // tile counts must fit int32 for the smallest tile
    if (*cells / (kBatchShapes[0].tile - 1) + bp->nbatch > (int64_t(1) << 30)) return WENOZN_EINVAL;
    return WENOZN_OK;
}

int default_shape() { return 3; }   // 512 interfaces x 256 threads

// Process-wide tuning table: the tile shape the tuner found fastest, keyed by what decides
// it (the device, the boundary's ghost map, and the binary orders of magnitude of the mean
// instance size and of the batch's total cell count; every batch is 1D Euler).  A step with
// shape = -1 uses the entry of its key, so a batch of a size class already tuned in this
// process is not timed again.
struct TuneKey {
    int dev, bc, mean_log2, total_log2;
    bool operator<(const TuneKey& o) const {
        return std::tie(dev, bc, mean_log2, total_log2) < std::tie(o.dev, o.bc, o.mean_log2, o.total_log2);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

int floor_log2(int64_t v) {
    int r = 0;
    while (v > 1) {
        v >>= 1;
        ++r;
    }
    return r;
}

TuneKey key_of(const wenozn_batch_params* bp, int64_t cells) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    return TuneKey{dev, bp->bc, floor_log2(cells / bp->nbatch), floor_log2(cells)};
}

// The shape a step uses: the caller's, else the table's entry for this batch, else the default.
int resolve_shape(const wenozn_batch_params* bp, int64_t cells) {
    if (bp->shape >= 0) return bp->shape;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key_of(bp, cells));
    return it != g_tuned.end() ? it->second : default_shape();
}

struct TileSizes { int v[kNumBatchShapes]; };

// Tile prefix counts of every shape: tile_off[s][b] = sum_{b' < b} ceil(n_b' / (tile_s - 1)).
__global__ void batch_tiles_kernel(const int64_t* off, int B, int32_t* tile_off, TileSizes tiles) {
    const int s = threadIdx.x;
    if (s >= kNumBatchShapes) return;
    const int per = tiles.v[s] - 1;
    int32_t acc = 0;
    int32_t* row = tile_off + size_t(s) * (B + 1);
    row[0] = 0;
    for (int b = 0; b < B; ++b) {
        const int64_t n = off[b + 1] - off[b];
        acc += int32_t((n + per - 1) / per);
        row[b + 1] = acc;
    }
}

struct Ptrs {
    Ctrl* ctrl;
    int64_t* off;
    int32_t* tile_off;
    double* dx;
    unsigned long long* alpha;
    double* dt;
    double* t;
    double* u1;
    double* u2;
};

Ptrs ptrs_of(void* ws, const BatchLayout& L) {
    char* b = static_cast<char*>(ws);
    Ptrs p;
    p.ctrl = reinterpret_cast<Ctrl*>(b + L.ctrl);
    p.off = reinterpret_cast<int64_t*>(b + L.off);
    p.tile_off = reinterpret_cast<int32_t*>(b + L.tile_off);
    p.dx = reinterpret_cast<double*>(b + L.dx);
    p.alpha = reinterpret_cast<unsigned long long*>(b + L.alpha);
    p.dt = reinterpret_cast<double*>(b + L.dt);
    p.t = reinterpret_cast<double*>(b + L.t);
    p.u1 = reinterpret_cast<double*>(b + L.u1);
    p.u2 = reinterpret_cast<double*>(b + L.u2);
    return p;
}

BatchArgs args_of(const wenozn_batch_params* bp, const Ptrs& p, int64_t cells, int shape) {
    BatchArgs a;
    std::memset(&a, 0, sizeof a);
    a.total = cells;
    a.B = bp->nbatch;
    a.off = p.off;
    a.tile_off = p.tile_off + size_t(shape) * (bp->nbatch + 1);
    a.dx = p.dx;
    a.alpha = p.alpha;
    a.dt = p.dt;
    a.t = p.t;
    a.status = &p.ctrl->status;
    a.bc = bp->bc;
    a.gamma = bp->gamma;
    a.eps4 = 4.0 * bp->eps;
    a.kappa = zn_kappa(bp->A);
    a.cfl = bp->cfl;
    a.t_final = bp->t_final;
    return a;
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 152;
    return sms > 0 ? sms : 152;
}

cudaError_t step_launches(const wenozn_batch_params* bp, const Ptrs& p, int64_t cells, double* U,
                          int shape, cudaStream_t s) {
    const int sms = sm_count();
    BatchArgs a = args_of(bp, p, cells, shape);
    const double* in[3] = {U, p.u1, p.u2};
    double* out[3] = {p.u1, p.u2, U};
    for (int st = 0; st < 3; ++st) {
        a.stage = st;
        a.Us = in[st];
        a.Un = U;
        a.out = out[st];
        cudaError_t e = launch_batch_stage(shape, a, sms, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

int32_t wenozn_batch_num_shapes(void) { return kNumBatchShapes; }

wenozn_status wenozn_batch_shape(int32_t shape, int32_t* tile, int32_t* threads) {
    if (shape < 0 || shape >= kNumBatchShapes || !tile || !threads) return WENOZN_EINVAL;
    *tile = kBatchShapes[shape].tile;
    *threads = kBatchShapes[shape].threads;
    return WENOZN_OK;
}

wenozn_status wenozn_batch_workspace_size(const wenozn_batch_params* bp, const int64_t* offsets,
                                          size_t* bytes) {
    int64_t cells = 0;
    wenozn_status st = check_batch(bp, offsets, &cells);
    if (st != WENOZN_OK) return st;
    if (!bytes) return WENOZN_EINVAL;
    *bytes = batch_layout(bp->nbatch, cells).total;
    return WENOZN_OK;
}

wenozn_status wenozn_batch_init(const wenozn_batch_params* bp, const int64_t* offsets, const double* dx,
                                const double* U, void* ws, size_t ws_bytes, void* stream) {
    int64_t cells = 0;
    wenozn_status st = check_batch(bp, offsets, &cells);
    if (st != WENOZN_OK) return st;
    if (!dx || !U || !ws || reinterpret_cast<uintptr_t>(ws) % kAlign) return WENOZN_EINVAL;
    for (int b = 0; b < bp->nbatch; ++b)
        if (!(std::isfinite(dx[b]) && dx[b] > 0.0)) return WENOZN_EINVAL;
    const BatchLayout L = batch_layout(bp->nbatch, cells);
    if (ws_bytes < L.total) return WENOZN_ENOMEM_WS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Ptrs p = ptrs_of(ws, L);
    TileSizes tiles;
    for (int i = 0; i < kNumBatchShapes; ++i) tiles.v[i] = kBatchShapes[i].tile;
    cudaError_t e = batch_configure();
    if (e == cudaSuccess) e = cudaMemsetAsync(p.ctrl, 0, sizeof(Ctrl), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p.off, offsets, size_t(bp->nbatch + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p.dx, dx, size_t(bp->nbatch) * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        batch_tiles_kernel<<<1, 32, 0, s>>>(p.off, bp->nbatch, p.tile_off, tiles);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        BatchArgs a = args_of(bp, p, cells, 0);
        a.Us = U;
        e = launch_batch_init(a, s);
    }
    // the host arrays may be released when this returns
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? WENOZN_OK : WENOZN_ECUDA;
}

wenozn_status wenozn_batch_rk3_step(const wenozn_batch_params* bp, const int64_t* offsets, double* U,
                                    void* ws, size_t ws_bytes, void* stream) {
    int64_t cells = 0;
    wenozn_status st = check_batch(bp, offsets, &cells);
    if (st != WENOZN_OK) return st;
    if (!U || !ws || reinterpret_cast<uintptr_t>(ws) % kAlign) return WENOZN_EINVAL;
    const BatchLayout L = batch_layout(bp->nbatch, cells);
    if (ws_bytes < L.total) return WENOZN_ENOMEM_WS;
    const int shape = resolve_shape(bp, cells);
    const Ptrs bptr = ptrs_of(ws, L);
    note_status(stream, &bptr.ctrl->status);
    cudaError_t e = step_launches(bp, bptr, cells, U, shape, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? WENOZN_OK : WENOZN_ECUDA;
}

wenozn_status wenozn_batch_tune(wenozn_batch_params* bp, const int64_t* offsets, double* U, void* ws,
                                size_t ws_bytes, int32_t steps, float* ms_per_step, void* stream) {
    int64_t cells = 0;
    wenozn_status st = check_batch(bp, offsets, &cells);
    if (st != WENOZN_OK) return st;
    if (!U || !ws || steps < 0 || reinterpret_cast<uintptr_t>(ws) % kAlign) return WENOZN_EINVAL;
    const BatchLayout L = batch_layout(bp->nbatch, cells);
    if (ws_bytes < L.total) return WENOZN_ENOMEM_WS;
    const TuneKey key = key_of(bp, cells);
    if (steps == 0) {            // the table's entry for this size class, if there is one
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            bp->shape = it->second;
            if (ms_per_step)
                for (int i = 0; i < kNumBatchShapes; ++i) ms_per_step[i] = 0.0f;
            return WENOZN_OK;
        }
    }
    if (steps == 0) steps = 2;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Ptrs p = ptrs_of(ws, L);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return WENOZN_ECUDA;
    }
    int best = -1;
    float best_ms = 0.0f;
    cudaError_t e = cudaSuccess;
    for (int shape = 0; shape < kNumBatchShapes && e == cudaSuccess; ++shape) {
        e = step_launches(bp, p, cells, U, shape, s);          // warm-up step
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int k = 0; k < steps && e == cudaSuccess; ++k) e = step_launches(bp, p, cells, U, shape, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        ms /= float(steps);
        if (ms_per_step) ms_per_step[shape] = ms;
        if (e == cudaSuccess && (best < 0 || ms < best_ms)) {
            best = shape;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return WENOZN_ECUDA;
    bp->shape = best;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[key] = best;
    return WENOZN_OK;
}

wenozn_status wenozn_batch_resolved_shape(const wenozn_batch_params* bp, const int64_t* offsets, int32_t* shape) {
    int64_t cells = 0;
    wenozn_status st = check_batch(bp, offsets, &cells);
    if (st != WENOZN_OK) return st;
    if (!shape) return WENOZN_EINVAL;
    *shape = resolve_shape(bp, cells);
    return WENOZN_OK;
}

wenozn_status wenozn_batch_state(void* ws, int32_t nbatch, const int64_t* offsets, double** t,
                                 double** dt, int32_t** status) {
    if (!ws || !offsets || nbatch < 1) return WENOZN_EINVAL;
    const BatchLayout L = batch_layout(nbatch, offsets[nbatch]);
    const Ptrs p = ptrs_of(ws, L);
    if (t) *t = p.t;
    if (dt) *dt = p.dt;
    if (status) *status = &p.ctrl->status;
    return WENOZN_OK;
}

}  // extern "C"
