// The fused kernel over a batch of independent domains (cases): the tiles
// {case, x block, row} of every active case in one launch, each tile with its
// own case's parameters and step counter; and the open-channel columns of
// every active case.  The device code is in k_stream_collide.cuh.
#include "k_stream_collide.cuh"

namespace gbm {

namespace {

// Batch of independent domains: persistent blocks walk the list of active
// tiles {case, x block, row} of all cases (case-major), each tile with its
// own case's parameters and step counter.
template <int P, int V, bool FORCE, bool LOCAL>
__global__ void __launch_bounds__(SC_BLOCK_X, 6)
    k_stream_collide_batch(const StepParams *__restrict__ cases, const int4 *__restrict__ tiles,
                           const int *__restrict__ ntiles) {
    const int n = *ntiles;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int4 tl = tiles[k];
        sc_tile<P, V, FORCE, LOCAL>(cases[tl.x], tl.y, tl.z);
    }
}

// The same tiles with one block per tile (grid = capacity of the list).
// FP32 with 4- or 8-byte words: at most 48 registers (10 blocks per SM, as
// the single-domain kernel), at the cost of a few bytes of spills.
template <int P, int V>
constexpr int tiles_min_blocks() { return (P == LBM_FP32_DEV && V <= 2) ? 10 : 6; }

template <int P, int V, bool FORCE, bool LOCAL>
__global__ void __launch_bounds__(SC_BLOCK_X, (tiles_min_blocks<P, V>()))
    k_stream_collide_tiles(const StepParams *__restrict__ cases, const int4 *__restrict__ tiles,
                           const int *__restrict__ ntiles) {
    if ((int)blockIdx.x >= *ntiles) return;
    const int4 tl = tiles[blockIdx.x];
    sc_tile<P, V, FORCE, LOCAL>(cases[tl.x], tl.y, tl.z);
}

// Open-channel columns of the active cases: one block per active case.
template <int P, bool FORCE>
__global__ void k_open_batch(const StepParams *__restrict__ cases, const int *__restrict__ active,
                             const int *__restrict__ nactive) {
    using R = typename Raw<P>::R;
    if ((int)blockIdx.x >= *nactive) return;
    const StepParams &p = cases[active[blockIdx.x]];
    if (p.L.bc_x != LBM_OPEN) return;
    const long long t = *p.t;
    R *f = static_cast<R *>((t & 1) ? p.f0 : p.f1);
    for (int y = threadIdx.x; y < p.L.ny; y += blockDim.x) open_row<P, FORCE>(p, f, y);
}

template <int P, int V, bool FORCE, bool LOCAL>
cudaError_t launch_scb(const BatchLaunch &b, cudaStream_t st) {
    static int per_sm = -1, sms = 0;
    if (per_sm < 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k_stream_collide_batch<P, V, FORCE, LOCAL>, SC_BLOCK_X, 0);
        if (e != cudaSuccess) return e;
    }
    if (b.persistent)
        k_stream_collide_batch<P, V, FORCE, LOCAL>
            <<<per_sm * sms, SC_BLOCK_X, 0, st>>>(b.cases, b.tiles, b.ntiles);
    else if (b.max_tiles > 0)
        k_stream_collide_tiles<P, V, FORCE, LOCAL>
            <<<b.max_tiles, SC_BLOCK_X, 0, st>>>(b.cases, b.tiles, b.ntiles);
    return cudaGetLastError();
}

template <int P, int V>
cudaError_t launch_scb_v(const BatchLaunch &b, cudaStream_t st) {
    if (b.force)
        return b.local ? launch_scb<P, V, true, true>(b, st) : launch_scb<P, V, true, false>(b, st);
    return b.local ? launch_scb<P, V, false, true>(b, st) : launch_scb<P, V, false, false>(b, st);
}

template <int P>
cudaError_t launch_scb_p(const BatchLaunch &b, cudaStream_t st) {
    constexpr int V16 = 16 / (int)sizeof(typename Raw<P>::R);
    switch (b.variant) {
        case 1: return launch_scb_v<P, V16 / 2>(b, st);
        case 2: return launch_scb_v<P, (V16 / 4 > 0 ? V16 / 4 : 1)>(b, st);
        default: return launch_scb_v<P, V16>(b, st);
    }
}

template <int P>
cudaError_t launch_ob(const BatchLaunch &b, int ncase, cudaStream_t st) {
    if (b.force) k_open_batch<P, true><<<ncase, 128, 0, st>>>(b.cases, b.active, b.nactive);
    else k_open_batch<P, false><<<ncase, 128, 0, st>>>(b.cases, b.active, b.nactive);
    return cudaGetLastError();
}

}  // namespace

int tile_nodes(int precision, int variant) {
    const int v16 = precision == LBM_FP64 ? 2 : (precision == LBM_FP32_DEV ? 4 : 8);
    const int v = variant == 1 ? v16 / 2 : (variant == 2 ? (v16 / 4 > 0 ? v16 / 4 : 1) : v16);
    return SC_BLOCK_X * v;
}

cudaError_t launch_stream_collide_batch(const BatchLaunch &b, cudaStream_t st) {
    switch (b.precision) {
        case LBM_FP64: return launch_scb_p<LBM_FP64>(b, st);
        case LBM_FP32_DEV: return launch_scb_p<LBM_FP32_DEV>(b, st);
        default: return launch_scb_p<LBM_FP16_DEV>(b, st);
    }
}

cudaError_t launch_open_batch(const BatchLaunch &b, int ncase, cudaStream_t st) {
    switch (b.precision) {
        case LBM_FP64: return launch_ob<LBM_FP64>(b, ncase, st);
        case LBM_FP32_DEV: return launch_ob<LBM_FP32_DEV>(b, ncase, st);
        default: return launch_ob<LBM_FP16_DEV>(b, ncase, st);
    }
}

}  // namespace gbm
