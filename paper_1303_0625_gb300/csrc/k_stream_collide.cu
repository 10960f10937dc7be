// Fused pull-advection + half-way bounce-back + BGK collision (Eq. 1-3, Eq. 8)
// on one domain: one block per tile (row y, SC_BLOCK_X * V nodes); and the
// open-channel columns pass.  The device code is in k_stream_collide.cuh.
#include "k_stream_collide.cuh"

namespace gbm {

namespace {

template <int P, int V, bool FORCE, bool LOCAL, bool WALLS, bool DEFER, int COLL = 0,
          bool BND = false>
__global__ void __launch_bounds__(SC_BLOCK_X) k_stream_collide(const StepParams p) {
    sc_tile<P, V, FORCE, LOCAL, false, WALLS, DEFER, COLL, BND>(p, blockIdx.x, blockIdx.y);
}

// With the per-node path deferred (variants 3-5), the nodes k_stream_collide
// leaves to the per-node update (update_node) are computed from the same
// populations after it, by k_boundary_update: one thread per node of the
// step's list of fluid nodes next to solids, then of the first and last
// columns and, where the vector path does not take them, of the wall rows.
// The force kernel of the step fills the list: it visits every fluid node
// with a link into its solid (one atomic per warp and list chunk).  The
// list's length is kept per step parity; the update kernel of step t clears
// the slot of step t + 1.  A node next to two disks is computed twice, with
// identical results.  Inline in the vector path these nodes run with one or
// two active lanes per warp; which way is faster depends on the workload (the
// autotuner measures both).
constexpr int BN_BLOCK = 256;

template <int P, bool FORCE, bool LOCAL>
__host__ __device__ long long boundary_edge_nodes(const Lattice &L) {
    long long n = L.nx > 1 ? 2LL * L.ny : (long long)L.ny;
    if (!walls_on_vector_path<P, LOCAL>() && L.bc_y == LBM_WALL && L.nx > 2) n += 2LL * (L.nx - 2);
    return n;
}

template <int P, bool FORCE, bool LOCAL, bool BND>
__global__ void __launch_bounds__(BN_BLOCK) k_boundary_update(const StepParams p) {
    using R = typename Raw<P>::R;
    const Lattice &L = p.L;
    const long long t = *p.t;
    const R *fin = static_cast<const R *>((t & 1) ? p.f1 : p.f0);
    R *fout = static_cast<R *>((t & 1) ? p.f0 : p.f1);
    const int nlist = (p.nsolid > 0 && p.bnd) ? min(p.bnd[t & 1], p.bnd_cap) : 0;
    const int ncol = L.nx > 1 ? 2 * L.ny : L.ny;
    const long long total = nlist + boundary_edge_nodes<P, FORCE, LOCAL>(L);
    for (long long e = (long long)blockIdx.x * BN_BLOCK + threadIdx.x; e < total;
         e += (long long)gridDim.x * BN_BLOCK) {
        int x, y;
        if (e < nlist) {
            const int k = p.bnd[2 + e];
            x = k % L.pitch;
            y = k / L.pitch;
        } else if (e < nlist + ncol) {
            const int c = (int)(e - nlist);
            y = L.nx > 1 ? c >> 1 : c;
            x = (L.nx > 1 && (c & 1)) ? L.nx - 1 : 0;
        } else {
            const int c = (int)(e - nlist - ncol), w = L.nx - 2;
            y = c < w ? 0 : L.ny - 1;
            x = 1 + (c < w ? c : c - w);
        }
        if (!(p.flags[cell_of(L, x, y)] & 1u))
            update_node<P, FORCE, LOCAL, false, 0, BND>(p, fin, fout, x, y);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && p.bnd) p.bnd[(t + 1) & 1] = 0;
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

template <int P, bool FORCE, bool LOCAL>
cudaError_t launch_update(const StepParams &p, cudaStream_t st);

// Walled domains (y walls) with rho_w = rho0 in FP32/FP64 take the kernel
// whose vector path also covers the wall rows.
template <int P, int V, bool FORCE, bool LOCAL, bool DEFER>
cudaError_t launch_sc(const StepParams &p, cudaStream_t st) {
    dim3 grid((p.L.nx + SC_BLOCK_X * V - 1) / (SC_BLOCK_X * V), p.L.ny);
    if (walls_on_vector_path<P, LOCAL>() && p.L.bc_y == LBM_WALL)
        k_stream_collide<P, V, FORCE, LOCAL, walls_on_vector_path<P, LOCAL>(), DEFER>
            <<<grid, SC_BLOCK_X, 0, st>>>(p);
    else
        k_stream_collide<P, V, FORCE, LOCAL, false, DEFER><<<grid, SC_BLOCK_X, 0, st>>>(p);
    cudaError_t e = cudaGetLastError();
    // with solids, the force kernel lists the nodes next to them and the
    // host launches the update after it (launch_deferred_update)
    if (e != cudaSuccess || !DEFER || p.list_by_forces) return e;
    return launch_update<P, FORCE, LOCAL>(p, st);
}

// The update kernel of the deferred per-node path, over the list of step t.
template <int P, bool FORCE, bool LOCAL>
cudaError_t launch_update(const StepParams &p, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const long long most = (p.nsolid > 0 ? p.bnd_cap : 0) + boundary_edge_nodes<P, FORCE, LOCAL>(p.L);
    long long blocks = (most + BN_BLOCK - 1) / BN_BLOCK;
    if (blocks > 8LL * sms) blocks = 8LL * sms;
    if (blocks < 1) blocks = 1;
    if (p.boundary == LBM_INTERPOLATED)
        k_boundary_update<P, FORCE, LOCAL, true><<<(unsigned)blocks, BN_BLOCK, 0, st>>>(p);
    else
        k_boundary_update<P, FORCE, LOCAL, false><<<(unsigned)blocks, BN_BLOCK, 0, st>>>(p);
    return cudaGetLastError();
}

template <int P, int V, bool DEFER>
cudaError_t launch_sc_v(const StepParams &p, cudaStream_t st) {
    const bool force = p.body_x != 0.0 || p.body_y != 0.0;
    const bool local = p.rho_w_mode == LBM_RHOW_LOCAL;
    if (force)
        return local ? launch_sc<P, V, true, true, DEFER>(p, st)
                     : launch_sc<P, V, true, false, DEFER>(p, st);
    return local ? launch_sc<P, V, false, true, DEFER>(p, st)
                 : launch_sc<P, V, false, false, DEFER>(p, st);
}

// Node widths per thread: variant 0 = one 16-byte word per population,
// variant 1 = 8 bytes, variant 2 = 4 bytes; variants 3-5 the same widths
// with the per-node path deferred to k_boundary_update.
// MRT: one launch shape, 8-byte words per population plane, slow nodes inline.
template <int P, bool LOCAL, bool BND>
cudaError_t launch_mrt_b(const StepParams &p, cudaStream_t st) {
    constexpr int V = 8 / (int)sizeof(typename Raw<P>::R) > 0 ? 8 / (int)sizeof(typename Raw<P>::R) : 1;
    dim3 grid((p.L.nx + SC_BLOCK_X * V - 1) / (SC_BLOCK_X * V), p.L.ny);
    if (walls_on_vector_path<P, LOCAL>() && p.L.bc_y == LBM_WALL)
        k_stream_collide<P, V, false, LOCAL, walls_on_vector_path<P, LOCAL>(), false, 1, BND>
            <<<grid, SC_BLOCK_X, 0, st>>>(p);
    else
        k_stream_collide<P, V, false, LOCAL, false, false, 1, BND><<<grid, SC_BLOCK_X, 0, st>>>(p);
    return cudaGetLastError();
}

template <int P, bool LOCAL>
cudaError_t launch_mrt(const StepParams &p, cudaStream_t st) {
    return p.boundary == LBM_INTERPOLATED ? launch_mrt_b<P, LOCAL, true>(p, st)
                                          : launch_mrt_b<P, LOCAL, false>(p, st);
}

template <int P>
cudaError_t launch_sc_p(const StepParams &p, cudaStream_t st) {
    if (p.collision == LBM_MRT)
        return p.rho_w_mode == LBM_RHOW_LOCAL ? launch_mrt<P, true>(p, st) : launch_mrt<P, false>(p, st);
    constexpr int V16 = 16 / (int)sizeof(typename Raw<P>::R);
    constexpr int V4 = V16 / 4 > 0 ? V16 / 4 : 1;
    // the interpolated boundary runs the per-node path in the deferred pass only
    switch (p.boundary == LBM_INTERPOLATED && p.sc_variant < 3 ? p.sc_variant + 3 : p.sc_variant) {
        case 1: return launch_sc_v<P, V16 / 2, false>(p, st);
        case 2: return launch_sc_v<P, V4, false>(p, st);
        case 3: return launch_sc_v<P, V16, true>(p, st);
        case 4: return launch_sc_v<P, V16 / 2, true>(p, st);
        case 5: return launch_sc_v<P, V4, true>(p, st);
        default: return launch_sc_v<P, V16, false>(p, st);
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

cudaError_t launch_deferred_update(const StepParams &p, cudaStream_t st) {
    const bool force = p.body_x != 0.0 || p.body_y != 0.0;
    const bool local = p.rho_w_mode == LBM_RHOW_LOCAL;
#define GBM_U(P)                                                                            \
    return force ? (local ? launch_update<P, true, true>(p, st) : launch_update<P, true, false>(p, st)) \
                 : (local ? launch_update<P, false, true>(p, st) : launch_update<P, false, false>(p, st))
    switch (p.precision) {
        case LBM_FP64: GBM_U(LBM_FP64);
        case LBM_FP32_DEV: GBM_U(LBM_FP32_DEV);
        default: GBM_U(LBM_FP16_DEV);
    }
#undef GBM_U
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
