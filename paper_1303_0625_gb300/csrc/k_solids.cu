// Per-solid kernels: momentum-exchange forces (Eq. 4-7), solid motion,
// re-rasterisation of moving disks, covered/fresh node handling (Sec. I and
// Sec. IV.B), plus initialisation and export kernels.
//
// Every per-solid kernel runs one block per solid over the bounding box of its
// disk, so the work per step scales with the solids' perimeter and area, not
// with the domain.  The fluid-solid links of solid s are enumerated inside its
// box from the node flags (bit j of a fluid node: x - e_j is solid or outside)
// and the owner map, in raster order of the box; per-thread FP64 partial sums
// are combined by a fixed warp-shuffle + shared-memory tree, so the force
// record is deterministic.
#include "lbm_internal.cuh"

namespace gbm {

namespace {

constexpr double PI = 3.14159265358979323846;

// Sum N doubles over the block; the result is valid in thread 0.
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N]) {
    __shared__ double sm[N][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < N; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; k++) sm[k][warp] = v[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int k = 0; k < N; k++) {
            v[k] = lane < nw ? sm[k][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        }
    }
}

__device__ __forceinline__ void atomic_min_u16(uint16_t *a, uint16_t v) {
    unsigned short old = *reinterpret_cast<volatile unsigned short *>(a);
    while (v < old) {
        unsigned short seen = atomicCAS(reinterpret_cast<unsigned short *>(a), old, v);
        if (seen == old) break;
        old = seen;
    }
}

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

__device__ __forceinline__ double net_weight(const StepParams &p, const DSolid &b) {
    const double M = b.rho_s * PI * b.r * b.r;
    const double g = sqrt(p.grav_x * p.grav_x + p.grav_y * p.grav_y);
    return fabs(1.0 - p.rho0 / b.rho_s) * M * g;
}

__device__ __forceinline__ double lub_mag(double kappa, double zeta, double gap) {
    if (gap >= zeta) return 0.0;
    const double q = (zeta - gap) / zeta;
    return kappa * q * q;
}

// Motion t -> t+1 of solid s; fg = Eq. 5 force and torque at t.
__device__ void move_solid(const StepParams &p, int s, long long t, const double *fg) {
    DSolid &b = p.S[s];
    if (b.motion == LBM_PRESCRIBED) {
        const double dt = (double)(t + 1 - b.ta);
        b.xn = __dadd_rn(b.xa, __dmul_rn(b.vx, dt));
        b.yn = __dadd_rn(b.ya, __dmul_rn(b.vy, dt));
        b.vxn = b.vx;
        b.vyn = b.vy;
        b.omn = b.om;
        return;
    }
    const Lattice &L = p.L;
    double flx = 0.0, fly = 0.0;
    if (p.lub > 0.0) {
        const double ka = net_weight(p, b);
        for (int q = 0; q < p.nsolid; q++) {
            if (q == s) continue;
            const DSolid &B = p.S[q];
            const double dx = min_image(b.x - B.x, L.nx, L.bc_x == LBM_PERIODIC);
            const double dy = min_image(b.y - B.y, L.ny, L.bc_y == LBM_PERIODIC);
            const double d = sqrt(dx * dx + dy * dy);
            const double kb = net_weight(p, B);
            const double m = lub_mag(ka > kb ? ka : kb, p.lub, d - b.r - B.r);
            if (m > 0.0 && d > 0.0) {
                flx += m * dx / d;
                fly += m * dy / d;
            }
        }
        if (L.bc_y == LBM_WALL) {
            fly += lub_mag(ka, p.lub, (b.y - b.r) + 0.5);
            fly -= lub_mag(ka, p.lub, ((double)L.ny - 0.5) - (b.y + b.r));
        }
        if (L.bc_x == LBM_WALL) {
            flx += lub_mag(ka, p.lub, (b.x - b.r) + 0.5);
            flx -= lub_mag(ka, p.lub, ((double)L.nx - 0.5) - (b.x + b.r));
        }
    }
    const double M = b.rho_s * PI * b.r * b.r;
    const double I = 0.5 * M * b.r * b.r;
    const double buoy = 1.0 - p.rho0 / b.rho_s;
    const double Fx = fg[0] + buoy * M * p.grav_x + flx;
    const double Fy = fg[1] + buoy * M * p.grav_y + fly;
    const double vx1 = b.vx + Fx / M, vy1 = b.vy + Fy / M;
    b.xn = b.x + 0.5 * (b.vx + vx1);
    b.yn = b.y + 0.5 * (b.vy + vy1);
    b.vxn = vx1;
    b.vyn = vy1;
    b.omn = b.om + fg[2] / I;
}

// ------------------------------------------------- forces at t (Eq. 4-7)

template <int P, bool LOCAL>
__global__ void __launch_bounds__(SOLID_BLOCK) k_forces(const StepParams p) {
    const int s = blockIdx.x;
    const Lattice &L = p.L;
    const long long t = *p.t;
    const void *fcur = (t & 1) ? p.f1 : p.f0;
    DSolid &b = p.S[s];
    if (!solid_ok(b)) {
        if (threadIdx.x == 0) atomicOr(p.status, 2);
        return;
    }
    const double X = b.x, Y = b.y, vx = b.vx, vy = b.vy, om = b.om;
    const Box bx = disk_box(X, Y, b.r, 1);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int c = threadIdx.x; c < bx.w * bx.h; c += blockDim.x) {
        int xf, yf;
        if (!locate(L, bx.x0 + c % bx.w, bx.y0 + c / bx.w, xf, yf)) continue;
        const long long k = cell_of(L, xf, yf);
        const uint16_t fl = p.flags[k];
        if ((fl & 1u) || !(fl & 0x1FEu)) continue;
        double rho_w = p.rho0;
        if (LOCAL) {
            rho_w = 0.0;
#pragma unroll
            for (int j = 0; j < 9; j++) rho_w += f64<P>(fcur, L.plane, j, k);
        }
#pragma unroll
        for (int i = 1; i < 9; i++) {
            if (!((fl >> opp(i)) & 1u)) continue;  // x_f + e_i not solid
            int xb, yb;
            if (!locate(L, xf + cx(i), yf + cy(i), xb, yb)) continue;
            if (p.owner[cell_of(L, xb, yb)] != s) continue;
            double ux, uy, dx, dy;  // boundary velocity at x_s = x_f + e_i / 2
            point_velocity(L, X, Y, vx, vy, om, (double)xf + 0.5 * cx(i),
                           (double)yf + 0.5 * cy(i), ux, uy, dx, dy);
            const double fi = f64<P>(fcur, L.plane, i, k);
            const double fbb = fi - 6.0 * wgt<double>(i) * rho_w * (cx(i) * ux + cy(i) * uy);
            // Eq. 4: e_i f_i - e_opp f_opp
            const double cmx = cx(i) * fi - cx(opp(i)) * fbb;
            const double cmy = cy(i) * fi - cy(opp(i)) * fbb;
            // Eq. 5: (e_i - v) f_i - (e_opp - v) f_opp
            const double gmx = (cx(i) - ux) * fi - (cx(opp(i)) - ux) * fbb;
            const double gmy = (cy(i) - uy) * fi - (cy(opp(i)) - uy) * fbb;
            acc[0] += cmx;                    // Eq. 6
            acc[1] += cmy;
            acc[2] += dx * cmy - dy * cmx;    // Eq. 7
            acc[3] += gmx;
            acc[4] += gmy;
            acc[5] += dx * gmy - dy * gmx;
        }
    }
    block_sum(acc);
    if (threadIdx.x == 0) {
        const long long slot = t % p.ring_len;
        double *rc = p.ring + (slot * 2 + 0) * p.nsolid * 3 + (long long)s * 3;
        double *rg = p.ring + (slot * 2 + 1) * p.nsolid * 3 + (long long)s * 3;
        double fg[3];
        for (int q = 0; q < 3; q++) {
            rc[q] = acc[q] + b.pend[q];
            fg[q] = acc[3 + q] + b.pend[q];
            rg[q] = fg[q];
            b.pend[q] = 0.0;
        }
        move_solid(p, s, t, fg);
    }
}

// ------------------------------------------------------------ remask

__global__ void __launch_bounds__(SOLID_BLOCK) k_remask_clear(const StepParams p) {
    const int s = p.moving[blockIdx.x];
    const DSolid &b = p.S[s];
    if (!solid_ok(b)) {
        if (threadIdx.x == 0) atomicOr(p.status, 2);
        return;
    }
    const Box bx = disk_box(b.x, b.y, b.r, 0);
    for (int c = threadIdx.x; c < bx.w * bx.h; c += blockDim.x) {
        int x, y;
        if (!locate(p.L, bx.x0 + c % bx.w, bx.y0 + c / bx.w, x, y)) continue;
        const long long k = cell_of(p.L, x, y);
        if (p.owner[k] == s) p.owner[k] = FLUID;
    }
}

// Rasterise solid s at (X, Y): lowest id wins.
__device__ __forceinline__ void stamp(const StepParams &p, int s, double X, double Y, double r) {
    const Box bx = disk_box(X, Y, r, 0);
    for (int c = threadIdx.x; c < bx.w * bx.h; c += blockDim.x) {
        const int iu = bx.x0 + c % bx.w, ju = bx.y0 + c / bx.w;
        if (!inside_disk(iu, ju, X, Y, r)) continue;
        int x, y;
        if (!locate(p.L, iu, ju, x, y)) continue;
        atomic_min_u16(p.owner + cell_of(p.L, x, y), (uint16_t)s);
    }
}

__global__ void __launch_bounds__(SOLID_BLOCK) k_remask_set(const StepParams p) {
    const DSolid &b = p.S[blockIdx.x];
    if (!solid_ok(b)) {
        if (threadIdx.x == 0) atomicOr(p.status, 2);
        return;
    }
    stamp(p, blockIdx.x, b.xn, b.yn, b.r);
}

__global__ void __launch_bounds__(SOLID_BLOCK) k_remask_flags(const StepParams p) {
    const DSolid &b = p.S[p.moving[blockIdx.x]];
    if (!solid_ok(b)) {
        if (threadIdx.x == 0) atomicOr(p.status, 2);
        return;
    }
    const Box bx = box_union(disk_box(b.x, b.y, b.r, 1), disk_box(b.xn, b.yn, b.r, 1));
    for (int c = threadIdx.x; c < bx.w * bx.h; c += blockDim.x) {
        int x, y;
        if (!locate(p.L, bx.x0 + c % bx.w, bx.y0 + c / bx.w, x, y)) continue;
        p.flags[cell_of(p.L, x, y)] = node_flags(p.L, p.owner, x, y);
    }
}

// A node that may feed a refill: fluid now and fluid before this step.
__device__ __forceinline__ bool usable(const StepParams &p, int x, int y, long long &k) {
    int xi, yi;
    if (!locate(p.L, x, y, xi, yi)) return false;
    k = cell_of(p.L, xi, yi);
    return p.owner[k] == FLUID && p.prev[k] == FLUID;
}

// Populations of a newborn node (Sec. IV.B): A1 second-order extrapolation
// along every direction with three old-fluid nodes, averaged; else A2 linear
// extrapolation; else A3 neighbour average; else equilibrium at rho0 and the
// solid's velocity at the node.
template <int P>
__device__ void refill_node(const StepParams &p, const void *f, int x, int y, const DSolid &b,
                            double (&out)[9]) {
    const long long pl = p.L.plane;
    double acc[9];
    int count;
    long long k1, k2, k3;
    if (p.refill <= LBM_REFILL_A1) {
        count = 0;
        for (int j = 0; j < 9; j++) acc[j] = 0.0;
        for (int i = 1; i < 9; i++) {
            if (!usable(p, x + cx(i), y + cy(i), k1)) continue;
            if (!usable(p, x + 2 * cx(i), y + 2 * cy(i), k2)) continue;
            if (!usable(p, x + 3 * cx(i), y + 3 * cy(i), k3)) continue;
            for (int j = 0; j < 9; j++)
                acc[j] += 3.0 * f64<P>(f, pl, j, k1) - 3.0 * f64<P>(f, pl, j, k2) +
                          f64<P>(f, pl, j, k3);
            count++;
        }
        if (count) {
            for (int j = 0; j < 9; j++) out[j] = acc[j] / count;
            return;
        }
    }
    if (p.refill <= LBM_REFILL_A2) {
        count = 0;
        for (int j = 0; j < 9; j++) acc[j] = 0.0;
        for (int i = 1; i < 9; i++) {
            if (!usable(p, x + cx(i), y + cy(i), k1)) continue;
            if (!usable(p, x + 2 * cx(i), y + 2 * cy(i), k2)) continue;
            for (int j = 0; j < 9; j++) acc[j] += 2.0 * f64<P>(f, pl, j, k1) - f64<P>(f, pl, j, k2);
            count++;
        }
        if (count) {
            for (int j = 0; j < 9; j++) out[j] = acc[j] / count;
            return;
        }
    }
    count = 0;
    for (int j = 0; j < 9; j++) acc[j] = 0.0;
    for (int i = 1; i < 9; i++) {
        if (!usable(p, x + cx(i), y + cy(i), k1)) continue;
        for (int j = 0; j < 9; j++) acc[j] += f64<P>(f, pl, j, k1);
        count++;
    }
    if (count) {
        for (int j = 0; j < 9; j++) out[j] = acc[j] / count;
        return;
    }
    double ux, uy, dx, dy;
    point_velocity(p.L, b.xn, b.yn, b.vxn, b.vyn, b.omn, (double)x, (double)y, ux, uy, dx, dy);
    const double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; i++) {
        const double eu = cx(i) * ux + cy(i) * uy;
        out[i] = p.rho0 * wgt<double>(i) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

// Covered nodes give their momentum to the solid; fresh nodes are refilled
// and take theirs from it.  Booked for the next force record.
template <int P>
__global__ void __launch_bounds__(SOLID_BLOCK) k_refill(const StepParams p) {
    const int s = p.moving[blockIdx.x];
    const Lattice &L = p.L;
    const long long t = *p.t;
    void *fnext = (t & 1) ? p.f0 : p.f1;
    DSolid &b = p.S[s];
    if (!solid_ok(b)) {
        if (threadIdx.x == 0) atomicOr(p.status, 2);
        return;
    }
    const Box bx = box_union(disk_box(b.x, b.y, b.r, 0), disk_box(b.xn, b.yn, b.r, 0));
    double acc[3] = {0, 0, 0};
    for (int c = threadIdx.x; c < bx.w * bx.h; c += blockDim.x) {
        int x, y;
        if (!locate(L, bx.x0 + c % bx.w, bx.y0 + c / bx.w, x, y)) continue;
        const long long k = cell_of(L, x, y);
        const uint16_t now = p.owner[k], was = p.prev[k];
        double sgn;
        if (was == FLUID && now == (uint16_t)s) {
            sgn = 1.0;  // covered
        } else if (was == (uint16_t)s && now == FLUID) {
            double nf[9];
            refill_node<P>(p, fnext, x, y, b, nf);
            for (int j = 0; j < 9; j++) put64<P>(fnext, L.plane, j, k, nf[j]);
            sgn = -1.0;  // fresh
        } else {
            continue;
        }
        double jx = 0.0, jy = 0.0;
        for (int j = 0; j < 9; j++) {
            const double v = f64<P>(fnext, L.plane, j, k);
            jx += cx(j) * v;
            jy += cy(j) * v;
        }
        double ux, uy, dx, dy;
        point_velocity(L, b.xn, b.yn, b.vxn, b.vyn, b.omn, (double)x, (double)y, ux, uy, dx, dy);
        acc[0] += sgn * jx;
        acc[1] += sgn * jy;
        acc[2] += sgn * (dx * jy - dy * jx);
    }
    block_sum(acc);
    if (threadIdx.x == 0) {
        b.pend[0] += acc[0];
        b.pend[1] += acc[1];
        b.pend[2] += acc[2];
    }
}

// prev := owner where it may have changed; the solid's state becomes t+1.
__global__ void __launch_bounds__(SOLID_BLOCK) k_remask_sync(const StepParams p) {
    const int s = p.moving[blockIdx.x];
    DSolid &b = p.S[s];
    if (!solid_ok(b)) {
        if (threadIdx.x == 0) {
            atomicOr(p.status, 2);
            if (blockIdx.x == 0) *p.t += 1;
        }
        return;
    }
    const Box bx = box_union(disk_box(b.x, b.y, b.r, 0), disk_box(b.xn, b.yn, b.r, 0));
    for (int c = threadIdx.x; c < bx.w * bx.h; c += blockDim.x) {
        int x, y;
        if (!locate(p.L, bx.x0 + c % bx.w, bx.y0 + c / bx.w, x, y)) continue;
        const long long k = cell_of(p.L, x, y);
        p.prev[k] = p.owner[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        b.x = b.xn;
        b.y = b.yn;
        b.vx = b.vxn;
        b.vy = b.vyn;
        b.om = b.omn;
        if (blockIdx.x == 0) *p.t += 1;
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

__global__ void k_flags_all(const StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= p.L.nx) return;
    p.flags[cell_of(p.L, x, y)] = node_flags(p.L, p.owner, x, y);
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
        p.prev[k] = p.owner[k];
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

dim3 cell_grid(const Lattice &L) { return dim3((L.nx + 127) / 128, L.ny); }

}  // namespace

// ------------------------------------------------------------ launchers

cudaError_t launch_forces(const StepParams &p, cudaStream_t st) {
    if (p.nsolid == 0) return cudaSuccess;
    const bool local = p.rho_w_mode == LBM_RHOW_LOCAL;
    switch (p.precision) {
        case LBM_FP64:
            if (local) k_forces<LBM_FP64, true><<<p.nsolid, SOLID_BLOCK, 0, st>>>(p);
            else k_forces<LBM_FP64, false><<<p.nsolid, SOLID_BLOCK, 0, st>>>(p);
            break;
        case LBM_FP32_DEV:
            if (local) k_forces<LBM_FP32_DEV, true><<<p.nsolid, SOLID_BLOCK, 0, st>>>(p);
            else k_forces<LBM_FP32_DEV, false><<<p.nsolid, SOLID_BLOCK, 0, st>>>(p);
            break;
        default:
            if (local) k_forces<LBM_FP16_DEV, true><<<p.nsolid, SOLID_BLOCK, 0, st>>>(p);
            else k_forces<LBM_FP16_DEV, false><<<p.nsolid, SOLID_BLOCK, 0, st>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_remask(const StepParams &p, cudaStream_t st) {
    if (p.nmoving == 0) {
        k_tick<<<1, 1, 0, st>>>(p);
        return cudaGetLastError();
    }
    k_remask_clear<<<p.nmoving, SOLID_BLOCK, 0, st>>>(p);
    k_remask_set<<<p.nsolid, SOLID_BLOCK, 0, st>>>(p);
    k_remask_flags<<<p.nmoving, SOLID_BLOCK, 0, st>>>(p);
    switch (p.precision) {
        case LBM_FP64: k_refill<LBM_FP64><<<p.nmoving, SOLID_BLOCK, 0, st>>>(p); break;
        case LBM_FP32_DEV: k_refill<LBM_FP32_DEV><<<p.nmoving, SOLID_BLOCK, 0, st>>>(p); break;
        default: k_refill<LBM_FP16_DEV><<<p.nmoving, SOLID_BLOCK, 0, st>>>(p);
    }
    k_remask_sync<<<p.nmoving, SOLID_BLOCK, 0, st>>>(p);
    return cudaGetLastError();
}

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
