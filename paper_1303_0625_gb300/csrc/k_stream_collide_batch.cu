// The fused kernel over a batch of independent domains (cases): the tiles
// {case, x block, first row} of every active case in one launch, each tile
// with its own case's parameters and step counter; open-channel columns are
// computed by the per-node path.  The device code is in k_stream_collide.cuh.
#include "k_stream_collide.cuh"

namespace gbm {

namespace {

// Batch of independent domains: persistent blocks walk the list of active
// tiles {case, x block, first row} of all cases (case-major), each tile
// (tile_h rows of SC_BLOCK_X * V nodes) with its own case's parameters and
// step counter.
template <int P, int V, bool FORCE, bool LOCAL>
__global__ void __launch_bounds__(SC_BLOCK_X, 6)
    k_stream_collide_batch(const StepParams *__restrict__ cases, const int4 *__restrict__ tiles,
                           const int *__restrict__ ntiles, int tile_h) {
    const int n = *ntiles;
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int4 tl = tiles[k];
        const StepParams &p = cases[tl.x];
        const int y1 = min(tl.z + tile_h, p.L.ny);
        for (int y = tl.z; y < y1; y++) sc_tile<P, V, FORCE, LOCAL, true, walls_on_vector_path<P, LOCAL>()>(p, tl.y, y);
    }
}

// The same tiles with one block per tile (grid = capacity of the list).
// FP32 with 4- or 8-byte words: at most 48 registers (10 blocks per SM, as
// the single-domain kernel), at the cost of a few bytes of spills.
template <int P, int V>
constexpr int tiles_min_blocks() { return (P == LBM_FP32_DEV && V <= 2) ? 10 : 6; }

template <int P, int V, bool FORCE, bool LOCAL, bool ROWS>
__global__ void __launch_bounds__(SC_BLOCK_X, (tiles_min_blocks<P, V>()))
    k_stream_collide_tiles(const StepParams *__restrict__ cases, const int4 *__restrict__ tiles,
                           const int *__restrict__ ntiles, int tile_h) {
    if ((int)blockIdx.x >= *ntiles) return;
    const int4 tl = tiles[blockIdx.x];
    const StepParams &p = cases[tl.x];
    if (!ROWS) {
        sc_tile<P, V, FORCE, LOCAL, true, walls_on_vector_path<P, LOCAL>()>(p, tl.y, tl.z);
        return;
    }
    const int y1 = min(tl.z + tile_h, p.L.ny);
    for (int y = tl.z; y < y1; y++) sc_tile<P, V, FORCE, LOCAL, true, walls_on_vector_path<P, LOCAL>()>(p, tl.y, y);
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
            <<<per_sm * sms, SC_BLOCK_X, 0, st>>>(b.cases, b.tiles, b.ntiles, b.tile_h);
    else if (b.max_tiles > 0 && b.tile_h == 1)
        k_stream_collide_tiles<P, V, FORCE, LOCAL, false>
            <<<b.max_tiles, SC_BLOCK_X, 0, st>>>(b.cases, b.tiles, b.ntiles, 1);
    else if (b.max_tiles > 0)
        k_stream_collide_tiles<P, V, FORCE, LOCAL, true>
            <<<b.max_tiles, SC_BLOCK_X, 0, st>>>(b.cases, b.tiles, b.ntiles, b.tile_h);
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

}  // namespace gbm
