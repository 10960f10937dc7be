// Fused pull-advection + half-way bounce-back + BGK collision (Eq. 1-3, Eq. 8)
// on one domain: one block per tile (row y, SC_BLOCK_X * V nodes); and the
// open-channel columns pass.  The device code is in k_stream_collide.cuh.
#include "k_stream_collide.cuh"

namespace gbm {

namespace {

template <int P, int V, bool FORCE, bool LOCAL, bool WALLS>
__global__ void __launch_bounds__(SC_BLOCK_X) k_stream_collide(const StepParams p) {
    sc_tile<P, V, FORCE, LOCAL, false, WALLS>(p, blockIdx.x, blockIdx.y);
}

// Open-channel columns of every row, on the populations of t+1.
template <int P, bool FORCE>
__global__ void k_open_columns(const StepParams p) {
    using R = typename Raw<P>::R;
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= p.L.ny) return;
    const long long t = *p.t;
    open_row<P, FORCE>(p, static_cast<R *>((t & 1) ? p.f0 : p.f1), y);
}

// Walled domains (y walls) with rho_w = rho0 in FP32/FP64 take the kernel
// whose vector path also covers the wall rows.
template <int P, int V, bool FORCE, bool LOCAL>
cudaError_t launch_sc(const StepParams &p, cudaStream_t st) {
    dim3 grid((p.L.nx + SC_BLOCK_X * V - 1) / (SC_BLOCK_X * V), p.L.ny);
    if (walls_on_vector_path<P, LOCAL>() && p.L.bc_y == LBM_WALL)
        k_stream_collide<P, V, FORCE, LOCAL, walls_on_vector_path<P, LOCAL>()>
            <<<grid, SC_BLOCK_X, 0, st>>>(p);
    else
        k_stream_collide<P, V, FORCE, LOCAL, false><<<grid, SC_BLOCK_X, 0, st>>>(p);
    return cudaGetLastError();
}

template <int P, int V>
cudaError_t launch_sc_v(const StepParams &p, cudaStream_t st) {
    const bool force = p.body_x != 0.0 || p.body_y != 0.0;
    const bool local = p.rho_w_mode == LBM_RHOW_LOCAL;
    if (force)
        return local ? launch_sc<P, V, true, true>(p, st) : launch_sc<P, V, true, false>(p, st);
    return local ? launch_sc<P, V, false, true>(p, st) : launch_sc<P, V, false, false>(p, st);
}

// Node widths per thread: variant 0 = one 16-byte word per population,
// variant 1 = 8 bytes, variant 2 = 4 bytes.
template <int P>
cudaError_t launch_sc_p(const StepParams &p, cudaStream_t st) {
    constexpr int V16 = 16 / (int)sizeof(typename Raw<P>::R);
    switch (p.sc_variant) {
        case 1: return launch_sc_v<P, V16 / 2>(p, st);
        case 2: return launch_sc_v<P, (V16 / 4 > 0 ? V16 / 4 : 1)>(p, st);
        default: return launch_sc_v<P, V16>(p, st);
    }
}

}  // namespace

cudaError_t launch_stream_collide(const StepParams &p, cudaStream_t st) {
    switch (p.precision) {
        case LBM_FP64: return launch_sc_p<LBM_FP64>(p, st);
        case LBM_FP32_DEV: return launch_sc_p<LBM_FP32_DEV>(p, st);
        default: return launch_sc_p<LBM_FP16_DEV>(p, st);
    }
}

cudaError_t launch_open_columns(const StepParams &p, cudaStream_t st) {
    if (p.L.bc_x != LBM_OPEN) return cudaSuccess;
    const bool force = p.body_x != 0.0 || p.body_y != 0.0;
    const dim3 grid((p.L.ny + 127) / 128);
    switch (p.precision) {
        case LBM_FP64:
            if (force) k_open_columns<LBM_FP64, true><<<grid, 128, 0, st>>>(p);
            else k_open_columns<LBM_FP64, false><<<grid, 128, 0, st>>>(p);
            break;
        case LBM_FP32_DEV:
            if (force) k_open_columns<LBM_FP32_DEV, true><<<grid, 128, 0, st>>>(p);
            else k_open_columns<LBM_FP32_DEV, false><<<grid, 128, 0, st>>>(p);
            break;
        default:
            if (force) k_open_columns<LBM_FP16_DEV, true><<<grid, 128, 0, st>>>(p);
            else k_open_columns<LBM_FP16_DEV, false><<<grid, 128, 0, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace gbm
