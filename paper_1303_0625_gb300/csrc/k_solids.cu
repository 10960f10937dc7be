// Set-up and export kernels: initial populations, node flags, rasterising an
// added disk, and copies of the state in FP64 for the caller.  The per-step
// work of the solids lives in k_solid_step.cu.
#include "lbm_internal.cuh"

namespace gbm {

namespace {

// bit 0: the node is solid; bit i (1..8): the node x - e_i is solid or
// beyond a non-periodic edge, i.e. population i arrives by bounce-back.
__device__ __forceinline__ uint16_t node_flags(const Lattice &L, const uint16_t *owner, int x,
                                               int y) {
    uint16_t f = owner[cell_of(L, x, y)] != FLUID ? 1u : 0u;
#pragma unroll
    for (int i = 1; i < 9; i++) {
        int xs, ys;
        if (!locate(L, x - cx(i), y - cy(i), xs, ys) || owner[cell_of(L, xs, ys)] != FLUID)
            f |= (uint16_t)(1u << i);
    }
    return f;
}

// Rasterise solid s at (X, Y): lowest id wins.
__device__ __forceinline__ void stamp(const StepParams &p, int s, double X, double Y, double r) {
    const Box bx = disk_box(X, Y, r, 0);
    const DiskTest inside(X, Y, r);
    for (int c = threadIdx.x; c < bx.w * bx.h; c += blockDim.x) {
        const int iu = bx.x0 + c % bx.w, ju = bx.y0 + c / bx.w;
        if (!inside(iu, ju)) continue;
        int x, y;
        if (!locate(p.L, iu, ju, x, y)) continue;
        atomic_min_u16(p.owner + cell_of(p.L, x, y), (uint16_t)s);
    }
}

__global__ void k_tick(const StepParams p) { *p.t += 1; }

// --------------------------------------------------------- initialisation

template <int P>
__global__ void k_init_populations(const StepParams p) {
    const Lattice &L = p.L;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= L.nx) return;
    double ux = p.u0x, uy = p.u0y;
    if (L.bc_x == LBM_OPEN) {
        const double h = (double)L.ny, yy = (double)y + 0.5;
        ux = 4.0 * p.umax * yy * (h - yy) / (h * h);
        uy = 0.0;
    }
    const double uu = ux * ux + uy * uy;
    const long long k = cell_of(L, x, y);
    for (int i = 0; i < 9; i++) {
        const double eu = cx(i) * ux + cy(i) * uy;
        const double f = p.rho0 * wgt<double>(i) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
        put64<P>(p.f0, L.plane, i, k, f);
        put64<P>(p.f1, L.plane, i, k, f);
    }
}

// Flags of every node; the row padding (nx <= x < pitch) is marked solid, so
// that the advection-collision kernel stores zeros there and never sends a
// padding node down the per-node path.
__global__ void k_flags_all(const StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= p.L.pitch) return;
    p.flags[cell_of(p.L, x, y)] = x < p.L.nx ? node_flags(p.L, p.owner, x, y) : (uint16_t)1u;
}

__global__ void __launch_bounds__(SOLID_BLOCK) k_stamp(const StepParams p, int s) {
    const DSolid &b = p.S[s];
    if (!solid_ok(b)) {
        if (threadIdx.x == 0) atomicOr(p.status, 2);
        return;
    }
    stamp(p, s, b.x, b.y, b.r);
}

__global__ void __launch_bounds__(SOLID_BLOCK) k_stamp_finish(const StepParams p, int s) {
    const DSolid &b = p.S[s];
    if (!solid_ok(b)) {
        if (threadIdx.x == 0) atomicOr(p.status, 2);
        return;
    }
    const Box bx = disk_box(b.x, b.y, b.r, 1);
    for (int c = threadIdx.x; c < bx.w * bx.h; c += blockDim.x) {
        int x, y;
        if (!locate(p.L, bx.x0 + c % bx.w, bx.y0 + c / bx.w, x, y)) continue;
        const long long k = cell_of(p.L, x, y);
        p.flags[k] = node_flags(p.L, p.owner, x, y);
    }
}

// ----------------------------------------------------------------- export

template <int P>
__global__ void k_export_populations(const StepParams p, double *out) {
    const Lattice &L = p.L;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= L.nx) return;
    const long long t = *p.t;
    const void *f = (t & 1) ? p.f1 : p.f0;
    const long long k = cell_of(L, x, y), n = (long long)L.nx * L.ny, o = (long long)y * L.nx + x;
    for (int i = 0; i < 9; i++) out[i * n + o] = f64<P>(f, L.plane, i, k);
}

template <int P>
__global__ void k_import_populations(const StepParams p, const double *in) {
    const Lattice &L = p.L;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= L.nx) return;
    const long long t = *p.t;
    void *f = (t & 1) ? p.f1 : p.f0;
    const long long k = cell_of(L, x, y), n = (long long)L.nx * L.ny, o = (long long)y * L.nx + x;
    for (int i = 0; i < 9; i++) put64<P>(f, L.plane, i, k, in[i * n + o]);
}

// Equilibrium initial state from a network prediction pred [3][ny][nx]
// (FP32): rho = 1 + R p0, u = U (p1, p2) at every fluid node (Eq. 8).
// With base, relative to the channel's Poiseuille flow (see lbm_nn.h).
template <int P>
__global__ void k_warm_start(const StepParams p, const float *pred, double U, double R, int base) {
    const Lattice &L = p.L;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= L.nx) return;
    const long long k = cell_of(L, x, y), n = (long long)L.nx * L.ny, o = (long long)y * L.nx + x;
    if (p.flags[k] & 1u) return;
    const long long t = *p.t;
    void *f = (t & 1) ? p.f1 : p.f0;
    double rho = 1.0 + R * (double)pred[o];
    double ux = U * (double)pred[n + o];
    const double uy = U * (double)pred[2 * n + o];
    if (base) {
        const double h = (double)L.ny, yy = (double)y + 0.5, nu = (p.tau - 0.5) / 3.0;
        ux += 4.0 * p.umax * yy * (h - yy) / (h * h);
        rho += p.rho0 - 1.0 + 24.0 * nu * p.umax * (double)(L.nx - 1 - x) / (h * h);
    }
    const double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; i++) {
        const double eu = cx(i) * ux + cy(i) * uy;
        put64<P>(f, L.plane, i, k, rho * wgt<double>(i) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
    }
}

// The same with the mass flux of every column made equal to the inlet's
// (open channel, walls in y): the steady flow carries the inlet's flux
// sum_y rho u_x through every column, and an error in it relaxes on the
// slowest scales of the channel.  One block per column x: rho and u_x of its
// fluid nodes as above (Poiseuille base), Q(x) = sum rho u_x and the inlet's
// Q_in = sum over column 0 of rho u_P (FP64, fixed tree), then
// u_x -> u_x Q_in / Q(x) and f = f^eq.
constexpr int WS_BLOCK = 128;

__device__ double block_sum_ws(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int k = 0; k < WS_BLOCK / 32; k++) t += sh[k];
    return t;
}

template <int P>
__global__ void __launch_bounds__(WS_BLOCK) k_warm_start_flux(const StepParams p, const float *pred,
                                                              double U, double R) {
    __shared__ double sh[WS_BLOCK / 32];
    const Lattice &L = p.L;
    const int x = blockIdx.x;
    const long long n = (long long)L.nx * L.ny;
    const long long t = *p.t;
    void *f = (t & 1) ? p.f1 : p.f0;
    const double h = (double)L.ny, nu = (p.tau - 0.5) / 3.0;
    auto rho_at = [&](int xx, int y) {
        return p.rho0 + R * (double)pred[(long long)y * L.nx + xx] +
               24.0 * nu * p.umax * (double)(L.nx - 1 - xx) / (h * h);
    };
    auto up_at = [&](int y) {
        const double yy = (double)y + 0.5;
        return 4.0 * p.umax * yy * (h - yy) / (h * h);
    };
    double q = 0.0, qin = 0.0;
    for (int y = threadIdx.x; y < L.ny; y += WS_BLOCK) {
        if (!(p.flags[cell_of(L, 0, y)] & 1u)) qin += rho_at(0, y) * up_at(y);
        if (!(p.flags[cell_of(L, x, y)] & 1u))
            q += rho_at(x, y) * (up_at(y) + U * (double)pred[n + (long long)y * L.nx + x]);
    }
    q = block_sum_ws(q, sh);
    qin = block_sum_ws(qin, sh);
    const double scale = q > 0.0 ? qin / q : 1.0;
    for (int y = threadIdx.x; y < L.ny; y += WS_BLOCK) {
        const long long k = cell_of(L, x, y), o = (long long)y * L.nx + x;
        if (p.flags[k] & 1u) continue;
        const double rho = rho_at(x, y);
        const double ux = (up_at(y) + U * (double)pred[n + o]) * scale;
        const double uy = U * (double)pred[2 * n + o];
        const double uu = ux * ux + uy * uy;
        for (int i = 0; i < 9; i++) {
            const double eu = cx(i) * ux + cy(i) * uy;
            put64<P>(f, L.plane, i, k, rho * wgt<double>(i) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
        }
    }
}

// Network input of a case, [8][ny][nx] floats: 0 the solid mask, 1 Re / 100,
// 2 log10(Re) / 2, 3 the signed distance to the nearest disk surface / 16
// (clipped to [-1, 4]), 4 the axial distance from that disk's centre in its
// radii / 8 (clipped to [-1, 4]; positive downstream), 5 the channel's
// parabola 4 y'(ny - y') / ny^2 (y' = y + 1/2), 6 x / nx, 7 y' / ny - 1/2.
// Geometry from the solid table, centres at the current time.
__global__ void k_case_features(const StepParams p, float re, float *in) {
    const Lattice &L = p.L;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= L.nx) return;
    const long long n = (long long)L.nx * L.ny, o = (long long)y * L.nx + x;
    float dmin = 1e30f, ax = 0.f;
    for (int s = 0; s < p.nsolid; s++) {
        const DSolid &b = p.S[s];
        const float dx = (float)((double)x - b.x), dy = (float)((double)y - b.y);
        const float r = sqrtf(b.r2f);
        const float d = sqrtf(dx * dx + dy * dy) - r;
        if (d < dmin) {
            dmin = d;
            ax = dx / (8.f * r);
        }
    }
    if (p.nsolid == 0) dmin = 64.f;
    const float h = (float)L.ny, yy = (float)y + 0.5f;
    in[o] = p.owner[cell_of(L, x, y)] != FLUID ? 1.f : 0.f;
    in[n + o] = re / 100.f;
    in[2 * n + o] = log10f(re) / 2.f;
    in[3 * n + o] = fminf(fmaxf(dmin / 16.f, -1.f), 4.f);
    in[4 * n + o] = fminf(fmaxf(ax, -1.f), 4.f);
    in[5 * n + o] = 4.f * yy * (h - yy) / (h * h);
    in[6 * n + o] = (float)x / (float)L.nx;
    in[7 * n + o] = yy / h - 0.5f;
}

__global__ void k_export_owner(const StepParams p, int32_t *out) {
    const Lattice &L = p.L;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= L.nx) return;
    const uint16_t s = p.owner[cell_of(L, x, y)];
    out[(long long)y * L.nx + x] = s == FLUID ? -1 : (int32_t)s;
}

template <int P>
__global__ void k_fields(const StepParams p, double *rho, double *ux, double *uy) {
    const Lattice &L = p.L;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= L.nx) return;
    const long long t = *p.t;
    const void *f = (t & 1) ? p.f1 : p.f0;
    const long long k = cell_of(L, x, y), o = (long long)y * L.nx + x;
    if (p.owner[k] != FLUID) {
        rho[o] = ux[o] = uy[o] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; i++) {
        const double v = f64<P>(f, L.plane, i, k);
        r += v;
        jx += cx(i) * v;
        jy += cy(i) * v;
    }
    rho[o] = r;
    ux[o] = (jx - 0.5 * p.body_x) / r;
    uy[o] = (jy - 0.5 * p.body_y) / r;
}

// bit i of mask[y][x]: fluid node x has a link along e_i (x + e_i solid).
__global__ void k_link_masks(const StepParams p, uint8_t *mask) {
    const Lattice &L = p.L;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= L.nx) return;
    uint8_t m = 0;
    if (p.owner[cell_of(L, x, y)] == FLUID) {
        for (int i = 1; i < 9; i++) {
            int xb, yb;
            if (locate(L, x + cx(i), y + cy(i), xb, yb) && p.owner[cell_of(L, xb, yb)] != FLUID)
                m |= (uint8_t)(1u << (i - 1));
        }
    }
    mask[(long long)y * L.nx + x] = m;
}

// covers the row padding too: (nx + 127) / 128 * 128 >= pitch = (nx + 63) / 64 * 64
dim3 cell_grid(const Lattice &L) { return dim3((L.nx + 127) / 128, L.ny); }

}  // namespace

// ------------------------------------------------------------ launchers

cudaError_t launch_tick(const StepParams &p, cudaStream_t st) {
    k_tick<<<1, 1, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_init_populations(const StepParams &p, cudaStream_t st) {
    switch (p.precision) {
        case LBM_FP64: k_init_populations<LBM_FP64><<<cell_grid(p.L), 128, 0, st>>>(p); break;
        case LBM_FP32_DEV: k_init_populations<LBM_FP32_DEV><<<cell_grid(p.L), 128, 0, st>>>(p); break;
        default: k_init_populations<LBM_FP16_DEV><<<cell_grid(p.L), 128, 0, st>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_flags_all(const StepParams &p, cudaStream_t st) {
    k_flags_all<<<cell_grid(p.L), 128, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_stamp_solid(const StepParams &p, int id, cudaStream_t st) {
    k_stamp<<<1, SOLID_BLOCK, 0, st>>>(p, id);
    k_stamp_finish<<<1, SOLID_BLOCK, 0, st>>>(p, id);
    return cudaGetLastError();
}

cudaError_t launch_export_populations(const StepParams &p, double *out, cudaStream_t st) {
    switch (p.precision) {
        case LBM_FP64: k_export_populations<LBM_FP64><<<cell_grid(p.L), 128, 0, st>>>(p, out); break;
        case LBM_FP32_DEV: k_export_populations<LBM_FP32_DEV><<<cell_grid(p.L), 128, 0, st>>>(p, out); break;
        default: k_export_populations<LBM_FP16_DEV><<<cell_grid(p.L), 128, 0, st>>>(p, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_import_populations(const StepParams &p, const double *in, cudaStream_t st) {
    switch (p.precision) {
        case LBM_FP64: k_import_populations<LBM_FP64><<<cell_grid(p.L), 128, 0, st>>>(p, in); break;
        case LBM_FP32_DEV: k_import_populations<LBM_FP32_DEV><<<cell_grid(p.L), 128, 0, st>>>(p, in); break;
        default: k_import_populations<LBM_FP16_DEV><<<cell_grid(p.L), 128, 0, st>>>(p, in);
    }
    return cudaGetLastError();
}

cudaError_t launch_warm_start(const StepParams &p, const float *pred, double u_scale,
                              double rho_scale, int base, cudaStream_t st) {
    if (base & 2) {  // the column flux made equal to the inlet's (with the Poiseuille base)
        switch (p.precision) {
            case LBM_FP64: k_warm_start_flux<LBM_FP64><<<p.L.nx, WS_BLOCK, 0, st>>>(p, pred, u_scale, rho_scale); break;
            case LBM_FP32_DEV: k_warm_start_flux<LBM_FP32_DEV><<<p.L.nx, WS_BLOCK, 0, st>>>(p, pred, u_scale, rho_scale); break;
            default: k_warm_start_flux<LBM_FP16_DEV><<<p.L.nx, WS_BLOCK, 0, st>>>(p, pred, u_scale, rho_scale);
        }
        return cudaGetLastError();
    }
    const dim3 g = cell_grid(p.L);
    switch (p.precision) {
        case LBM_FP64: k_warm_start<LBM_FP64><<<g, 128, 0, st>>>(p, pred, u_scale, rho_scale, base); break;
        case LBM_FP32_DEV: k_warm_start<LBM_FP32_DEV><<<g, 128, 0, st>>>(p, pred, u_scale, rho_scale, base); break;
        default: k_warm_start<LBM_FP16_DEV><<<g, 128, 0, st>>>(p, pred, u_scale, rho_scale, base);
    }
    return cudaGetLastError();
}

cudaError_t launch_case_features(const StepParams &p, double re, float *in, cudaStream_t st) {
    k_case_features<<<cell_grid(p.L), 128, 0, st>>>(p, (float)re, in);
    return cudaGetLastError();
}

cudaError_t launch_export_owner(const StepParams &p, int32_t *out, cudaStream_t st) {
    k_export_owner<<<cell_grid(p.L), 128, 0, st>>>(p, out);
    return cudaGetLastError();
}

cudaError_t launch_fields(const StepParams &p, double *rho, double *ux, double *uy,
                          cudaStream_t st) {
    switch (p.precision) {
        case LBM_FP64: k_fields<LBM_FP64><<<cell_grid(p.L), 128, 0, st>>>(p, rho, ux, uy); break;
        case LBM_FP32_DEV: k_fields<LBM_FP32_DEV><<<cell_grid(p.L), 128, 0, st>>>(p, rho, ux, uy); break;
        default: k_fields<LBM_FP16_DEV><<<cell_grid(p.L), 128, 0, st>>>(p, rho, ux, uy);
    }
    return cudaGetLastError();
}

cudaError_t launch_link_masks(const StepParams &p, uint8_t *mask, cudaStream_t st) {
    k_link_masks<<<cell_grid(p.L), 128, 0, st>>>(p, mask);
    return cudaGetLastError();
}

}  // namespace gbm
