// Per-solid work of one step, in a single cooperative launch after the
// advection-collision kernel of step t:
//
//   A  clear:   nodes of the old disk that the new disk leaves, owner s -> fluid
//   B  set:     nodes of the new disk, owner := lowest id covering them
//   C  changes: on the ring (old disk XOR new disk): node flags of every node
//               whose solidity changed and of its 8 neighbours; covered nodes
//               give their momentum to the solid; fresh (newborn) nodes are
//               refilled by extrapolation (Sec. IV.B) and take theirs from it
//   D  sync:    prev := owner on the ring; the solid's state becomes t+1
//   F  forces:  momentum exchange on every fluid-solid link at t+1 (Eq. 4 and
//               Eq. 5, summed by Eq. 6 and Eq. 7) plus the booked momenta,
//               written to the force history; motion t+1 -> t+2
//
// Phases A-D run only when some solid translates.  One warp owns one solid
// in a phase (solids are looped over when there are more solids than warps);
// phases are separated by a grid-wide barrier whose wait is bounded (status
// bit 2 and an early exit instead of a hang).  Work per solid follows its
// perimeter: every loop walks the disk's bounding box with an FP32 distance
// prefilter and touches memory only on the ring or the link annulus.
//
// Precision: in the FP32/FP16 modes the per-link products are evaluated in
// FP32 and summed per lane over one round of links; all accumulation across
// rounds and lanes (the force and torque reduction) is FP64.  The FP64 mode
// evaluates everything in FP64.
#include "lbm_internal.cuh"

namespace gbm {

namespace {

constexpr int SW_BLOCK = 256;
constexpr int WARPS = SW_BLOCK / 32;
constexpr int CELLS_PER_LANE = 8;
constexpr int ROUND = 32 * CELLS_PER_LANE;  // box cells per warp round
constexpr int QMAX = 8 * ROUND;             // at most 8 links per node
constexpr long long SPIN_LIMIT = 1ll << 24; // polls of about 64 ns: roughly one second
constexpr double PI = 3.14159265358979323846;

// ------------------------------------------------------------- barrier

// Grid-wide barrier for a cooperative launch.  Returns false (and raises
// status bit 2) if the other blocks did not arrive within SPIN_LIMIT polls.
__device__ bool grid_sync(const StepParams &p) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = p.bar + 1;
        const unsigned int g = *gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(p.bar, 1u) + 1u;
        ok = 1;
        if (arrived == gridDim.x) {
            atomicExch(p.bar, 0u);
            __threadfence();
            atomicAdd(p.bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*gen == g) {
                if (++spins > SPIN_LIMIT) {
                    atomicOr(p.status, 4);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// ------------------------------------------------------------- helpers

template <int N>
__device__ __forceinline__ void warp_sum(double (&v)[N]) {
#pragma unroll
    for (int k = 0; k < N; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
}

__device__ __forceinline__ int warp_exclusive_scan(int v, int &total) {
    const int lane = threadIdx.x & 31;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += n;
    }
    total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - v;
}

// Set or clear one bit of a 16-bit flags word atomically.
__device__ __forceinline__ void flag_bit(uint16_t *flags, long long k, int bit, bool on) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(flags + k);
    unsigned int *w = reinterpret_cast<unsigned int *>(a & ~uintptr_t(3));
    const unsigned int m = (1u << bit) << ((a & 2) ? 16 : 0);
    if (on) atomicOr(w, m);
    else atomicAnd(w, ~m);
}

// Box cell c -> unwrapped node coordinates.
__device__ __forceinline__ void box_cell(const Box &bx, int c, int &iu, int &ju) {
    ju = bx.y0 + c / bx.w;
    iu = bx.x0 + c - (ju - bx.y0) * bx.w;
}

// Population f_i of cell k in the link-math precision C.
template <int P>
__device__ __forceinline__ typename Prec<P>::C pop(const void *f, long long plane, int i,
                                                   long long k) {
    using C = typename Prec<P>::C;
    using S = typename Prec<P>::S;
    C v = (C)ldc(static_cast<const S *>(f) + (long long)i * plane + k);
    if (Prec<P>::dev) v += wgt<C>(i);
    return v;
}

// ------------------------------------------------------- phases A, B, D

__device__ void phase_clear(const StepParams &p, int s, int lane) {
    const DSolid &b = p.S[s];
    const DiskTest in0(b.x, b.y, b.r), in1(b.xn, b.yn, b.r);
    const Box bx = disk_box(b.x, b.y, b.r, 0);
    for (int c = lane; c < bx.w * bx.h; c += 32) {
        int iu, ju, x, y;
        box_cell(bx, c, iu, ju);
        if (!in0(iu, ju) || in1(iu, ju)) continue;
        if (!locate(p.L, iu, ju, x, y)) continue;
        const long long k = cell_of(p.L, x, y);
        if (p.owner[k] == (uint16_t)s) p.owner[k] = FLUID;
    }
}

__device__ void phase_set(const StepParams &p, int s, int lane) {
    const DSolid &b = p.S[s];
    const DiskTest in1(b.xn, b.yn, b.r);
    const Box bx = disk_box(b.xn, b.yn, b.r, 0);
    for (int c = lane; c < bx.w * bx.h; c += 32) {
        int iu, ju, x, y;
        box_cell(bx, c, iu, ju);
        if (!in1(iu, ju)) continue;
        if (!locate(p.L, iu, ju, x, y)) continue;
        uint16_t *o = p.owner + cell_of(p.L, x, y);
        if (*o > (uint16_t)s) atomic_min_u16(o, (uint16_t)s);
    }
}

__device__ void phase_sync(const StepParams &p, int s, int lane) {
    DSolid &b = p.S[s];
    const DiskTest in0(b.x, b.y, b.r), in1(b.xn, b.yn, b.r);
    const Box bx = box_union(disk_box(b.x, b.y, b.r, 0), disk_box(b.xn, b.yn, b.r, 0));
    for (int c = lane; c < bx.w * bx.h; c += 32) {
        int iu, ju, x, y;
        box_cell(bx, c, iu, ju);
        if (in0(iu, ju) == in1(iu, ju)) continue;
        if (!locate(p.L, iu, ju, x, y)) continue;
        const long long k = cell_of(p.L, x, y);
        if (p.prev[k] != p.owner[k]) p.prev[k] = p.owner[k];
    }
    __syncwarp();
    if (lane == 0) {
        b.x = b.xn;
        b.y = b.yn;
        b.xw = b.xnw;
        b.yw = b.ynw;
        b.vx = b.vxn;
        b.vy = b.vyn;
        b.om = b.omn;
        b.vxf = (float)b.vxn;
        b.vyf = (float)b.vyn;
        b.omf = (float)b.omn;
    }
}

// ------------------------------------------------------------ phase C

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
// solid's velocity at the node.  Works in the storage convention (f_i or
// f_i - w_i), which is linear, so extrapolation commutes with it.
template <int P>
__device__ void refill_node(const StepParams &p, const void *f, int x, int y, const DSolid &b,
                            typename Prec<P>::C (&out)[9]) {
    using C = typename Prec<P>::C;
    using S = typename Prec<P>::S;
    const S *fs = static_cast<const S *>(f);
    const long long pl = p.L.plane;
    C acc[9];
    int count;
    long long k1, k2, k3;
    if (p.refill <= LBM_REFILL_A1) {
        count = 0;
#pragma unroll
        for (int j = 0; j < 9; j++) acc[j] = 0;
        for (int i = 1; i < 9; i++) {
            if (!usable(p, x + cx(i), y + cy(i), k1)) continue;
            if (!usable(p, x + 2 * cx(i), y + 2 * cy(i), k2)) continue;
            if (!usable(p, x + 3 * cx(i), y + 3 * cy(i), k3)) continue;
#pragma unroll
            for (int j = 0; j < 9; j++)
                acc[j] += (C)3 * (C)ldc(fs + j * pl + k1) - (C)3 * (C)ldc(fs + j * pl + k2) +
                          (C)ldc(fs + j * pl + k3);
            count++;
        }
        if (count) {
#pragma unroll
            for (int j = 0; j < 9; j++) out[j] = acc[j] / (C)count;
            return;
        }
    }
    if (p.refill <= LBM_REFILL_A2) {
        count = 0;
#pragma unroll
        for (int j = 0; j < 9; j++) acc[j] = 0;
        for (int i = 1; i < 9; i++) {
            if (!usable(p, x + cx(i), y + cy(i), k1)) continue;
            if (!usable(p, x + 2 * cx(i), y + 2 * cy(i), k2)) continue;
#pragma unroll
            for (int j = 0; j < 9; j++)
                acc[j] += (C)2 * (C)ldc(fs + j * pl + k1) - (C)ldc(fs + j * pl + k2);
            count++;
        }
        if (count) {
#pragma unroll
            for (int j = 0; j < 9; j++) out[j] = acc[j] / (C)count;
            return;
        }
    }
    count = 0;
#pragma unroll
    for (int j = 0; j < 9; j++) acc[j] = 0;
    for (int i = 1; i < 9; i++) {
        if (!usable(p, x + cx(i), y + cy(i), k1)) continue;
#pragma unroll
        for (int j = 0; j < 9; j++) acc[j] += (C)ldc(fs + j * pl + k1);
        count++;
    }
    if (count) {
#pragma unroll
        for (int j = 0; j < 9; j++) out[j] = acc[j] / (C)count;
        return;
    }
    double ux, uy, dx, dy;
    point_velocity(p.L, b.xn, b.yn, b.vxn, b.vyn, b.omn, (double)x, (double)y, ux, uy, dx, dy);
    const double uu = ux * ux + uy * uy;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const double eu = cx(i) * ux + cy(i) * uy;
        const double fe = p.rho0 * wgt<double>(i) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
        out[i] = (C)(Prec<P>::dev ? fe - wgt<double>(i) : fe);
    }
}

template <int P>
__device__ void phase_changes(const StepParams &p, int s, int lane, long long t1, void *fnew) {
    using C = typename Prec<P>::C;
    using S = typename Prec<P>::S;
    DSolid &b = p.S[s];
    const Lattice &L = p.L;
    const DiskTest in0(b.x, b.y, b.r), in1(b.xn, b.yn, b.r);
    const Box bx = box_union(disk_box(b.x, b.y, b.r, 0), disk_box(b.xn, b.yn, b.r, 0));
    double acc[3] = {0.0, 0.0, 0.0};
    for (int c = lane; c < bx.w * bx.h; c += 32) {
        int iu, ju, x, y;
        box_cell(bx, c, iu, ju);
        if (in0(iu, ju) == in1(iu, ju)) continue;
        if (!locate(L, iu, ju, x, y)) continue;
        const long long k = cell_of(L, x, y);
        const uint16_t now = p.owner[k], was = p.prev[k];
        const bool sn = now != FLUID, sw = was != FLUID;
        if (sn != sw) {
            // bit 0 of the node, bit i of the neighbour x + e_i
            flag_bit(p.flags, k, 0, sn);
#pragma unroll
            for (int i = 1; i < 9; i++) {
                int xn, yn;
                if (locate(L, x + cx(i), y + cy(i), xn, yn)) flag_bit(p.flags, cell_of(L, xn, yn), i, sn);
            }
        }
        double sgn;
        if (!sw && now == (uint16_t)s) {
            sgn = 1.0;  // covered: its momentum goes to the solid
        } else if (was == (uint16_t)s && !sn) {
            C nf[9];
            refill_node<P>(p, fnew, x, y, b, nf);
#pragma unroll
            for (int j = 0; j < 9; j++) st(static_cast<S *>(fnew) + j * L.plane + k, nf[j]);
            sgn = -1.0;  // fresh: the solid gives it its momentum
        } else {
            continue;
        }
        double jx = 0.0, jy = 0.0;
#pragma unroll
        for (int j = 0; j < 9; j++) {
            const double v = f64<P>(fnew, L.plane, j, k);
            jx += cx(j) * v;
            jy += cy(j) * v;
        }
        double ux, uy, dx, dy;
        point_velocity(L, b.xn, b.yn, b.vxn, b.vyn, b.omn, (double)x, (double)y, ux, uy, dx, dy);
        acc[0] += sgn * jx;
        acc[1] += sgn * jy;
        acc[2] += sgn * (dx * jy - dy * jx);
    }
    warp_sum(acc);
    if (lane == 0) {
        b.pend[0] = acc[0];
        b.pend[1] = acc[1];
        b.pend[2] = acc[2];
        b.pend_t = t1;
    }
}

// ------------------------------------------------------------ phase F

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

// Motion tf -> tf+1 of solid s; fg = Eq. 5 force and torque at tf.
__device__ void move_solid(const StepParams &p, int s, long long tf, const double *fg) {
    DSolid &b = p.S[s];
    const Lattice &L = p.L;
    if (b.motion == LBM_PRESCRIBED) {
        const double dt = (double)(tf + 1 - b.ta);
        b.xn = __dadd_rn(b.xa, __dmul_rn(b.vx, dt));
        b.yn = __dadd_rn(b.ya, __dmul_rn(b.vy, dt));
        b.xnw = wrap_coord(b.xn, L.nx, L.bc_x == LBM_PERIODIC);
        b.ynw = wrap_coord(b.yn, L.ny, L.bc_y == LBM_PERIODIC);
        b.vxn = b.vx;
        b.vyn = b.vy;
        b.omn = b.om;
        return;
    }
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
    b.xnw = wrap_coord(b.xn, L.nx, L.bc_x == LBM_PERIODIC);
    b.ynw = wrap_coord(b.yn, L.ny, L.bc_y == LBM_PERIODIC);
    b.vxn = vx1;
    b.vyn = vy1;
    b.omn = b.om + fg[2] / I;
}

// Forces at time tf from the populations f of time tf (Eq. 4-7).
template <int P, bool LOCAL>
__device__ void phase_forces(const StepParams &p, int s, int lane, long long tf, const void *f,
                             uint16_t *queue) {
    using C = typename Prec<P>::C;
    DSolid &b = p.S[s];
    const Lattice &L = p.L;
    const double X = b.x, Y = b.y;
    const int xi = (int)floor(X), yi = (int)floor(Y);
    const float fx = (float)(X - xi), fy = (float)(Y - yi);
    const float r = (float)b.r;
    const float lo2 = (r - 0.01f) * (r - 0.01f), hi2 = (r + 1.5f) * (r + 1.5f);
    const C vx = pick<C>(b.vx, b.vxf), vy = pick<C>(b.vy, b.vyf), om = pick<C>(b.om, b.omf);
    const C rho0 = pick<C>(p.rho0, p.rho0_f);
    const Box bx = disk_box(X, Y, b.r, 1);
    const int n = bx.w * bx.h;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int base = 0; base < n; base += ROUND) {
        // link masks of this lane's cells in the round (8 bits per cell)
        unsigned long long masks = 0;
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < CELLS_PER_LANE; q++) {
            const int c = base + q * 32 + lane;
            if (c >= n) continue;
            int iu, ju, x, y;
            box_cell(bx, c, iu, ju);
            const float dx = (float)(iu - xi) - fx, dy = (float)(ju - yi) - fy;
            const float d2 = dx * dx + dy * dy;
            if (d2 <= lo2 || d2 > hi2) continue;  // outside the link annulus
            if (!locate(L, iu, ju, x, y)) continue;
            const uint16_t fl = p.flags[cell_of(L, x, y)];
            if ((fl & 1u) || !(fl & 0x1FEu)) continue;
            unsigned int m = 0;
#pragma unroll
            for (int i = 1; i < 9; i++) {
                if (!((fl >> opp(i)) & 1u)) continue;  // x_f + e_i not solid
                int xb, yb;
                if (!locate(L, x + cx(i), y + cy(i), xb, yb)) continue;
                if (p.owner[cell_of(L, xb, yb)] == (uint16_t)s) m |= 1u << (i - 1);
            }
            masks |= (unsigned long long)m << (8 * q);
            cnt += __popc(m);
        }
        int total;
        int off = warp_exclusive_scan(cnt, total);
        if (total == 0) continue;
#pragma unroll
        for (int q = 0; q < CELLS_PER_LANE; q++) {
            unsigned int m = (unsigned int)(masks >> (8 * q)) & 0xFFu;
            while (m) {
                const int i = __ffs(m);
                m &= m - 1;
                queue[off++] = (uint16_t)(((q * 32 + lane) << 3) | (i - 1));
            }
        }
        __syncwarp();
        C part[6] = {0, 0, 0, 0, 0, 0};
        for (int e = lane; e < total; e += 32) {
            const int code = queue[e];
            const int i = (code & 7) + 1;
            int iu, ju, x, y;
            box_cell(bx, base + (code >> 3), iu, ju);
            locate(L, iu, ju, x, y);
            const long long k = cell_of(L, x, y);
            C rho_w = rho0;
            if (LOCAL) {
                rho_w = 0;
#pragma unroll
                for (int j = 0; j < 9; j++) rho_w += pop<P>(f, L.plane, j, k);
            }
            // x_s = x_f + e_i / 2 relative to R, from the unwrapped box coordinate
            C dx, dy;
            if (Prec<P>::dev) {
                dx = (C)(iu - xi) + (C)(0.5f * cx(i)) - (C)fx;
                dy = (C)(ju - yi) + (C)(0.5f * cy(i)) - (C)fy;
            } else {
                dx = (C)(((double)iu + 0.5 * cx(i)) - X);
                dy = (C)(((double)ju + 0.5 * cy(i)) - Y);
            }
            const C ux = vx - om * dy, uy = vy + om * dx;
            const C fi = pop<P>(f, L.plane, i, k);
            const C fbb = fi - (C)6 * wgt<C>(i) * rho_w * ((C)cx(i) * ux + (C)cy(i) * uy);
            // Eq. 4: e_i f_i - e_opp f_opp;  Eq. 5: (e_i - v) f_i - (e_opp - v) f_opp
            const C cmx = (C)cx(i) * fi - (C)cx(opp(i)) * fbb;
            const C cmy = (C)cy(i) * fi - (C)cy(opp(i)) * fbb;
            const C gmx = ((C)cx(i) - ux) * fi - ((C)cx(opp(i)) - ux) * fbb;
            const C gmy = ((C)cy(i) - uy) * fi - ((C)cy(opp(i)) - uy) * fbb;
            part[0] += cmx;
            part[1] += cmy;
            part[2] += dx * cmy - dy * cmx;
            part[3] += gmx;
            part[4] += gmy;
            part[5] += dx * gmy - dy * gmx;
        }
#pragma unroll
        for (int q = 0; q < 6; q++) acc[q] += (double)part[q];
        __syncwarp();
    }
    warp_sum(acc);
    if (lane == 0) {
        const bool booked = b.pend_t == tf;
        const long long slot = tf % p.ring_len;
        double *rc = p.ring + (slot * 2 + 0) * p.nsolid * 3 + (long long)s * 3;
        double *rg = p.ring + (slot * 2 + 1) * p.nsolid * 3 + (long long)s * 3;
        double fg[3];
        for (int q = 0; q < 3; q++) {
            const double pb = booked ? b.pend[q] : 0.0;
            rc[q] = acc[q] + pb;
            fg[q] = acc[3 + q] + pb;
            rg[q] = fg[q];
        }
        move_solid(p, s, tf, fg);
    }
}

// ------------------------------------------------------------- kernel

template <int P, bool LOCAL>
__global__ void __launch_bounds__(SW_BLOCK) k_solids_step(const StepParams p, int mode) {
    __shared__ uint16_t queue[WARPS][QMAX];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * WARPS + wib, nw = gridDim.x * WARPS;
    const long long t = *p.t;
    const bool adv = (mode & SOLIDS_ADVANCE) != 0;
    const long long tf = adv ? t + 1 : t;
    void *ff = (tf & 1) ? p.f1 : p.f0;  // populations of time tf
    if (mode & SOLIDS_REMASK) {
        for (int m = gw; m < p.nmoving; m += nw) {
            const int s = p.moving[m];
            if (solid_ok(p.S[s])) phase_clear(p, s, lane);
            else if (lane == 0) atomicOr(p.status, 2);
        }
        grid_sync(p);
        for (int s = gw; s < p.nsolid; s += nw)
            if (solid_ok(p.S[s])) phase_set(p, s, lane);
        grid_sync(p);
        for (int m = gw; m < p.nmoving; m += nw) {
            const int s = p.moving[m];
            if (solid_ok(p.S[s])) phase_changes<P>(p, s, lane, tf, ff);
        }
        grid_sync(p);
        for (int m = gw; m < p.nmoving; m += nw) {
            const int s = p.moving[m];
            if (solid_ok(p.S[s])) phase_sync(p, s, lane);
        }
        grid_sync(p);
    }
    for (int s = gw; s < p.nsolid; s += nw) {
        if (solid_ok(p.S[s])) phase_forces<P, LOCAL>(p, s, lane, tf, ff, queue[wib]);
        else if (lane == 0) atomicOr(p.status, 2);
    }
    if (adv) {
        grid_sync(p);
        if (blockIdx.x == 0 && threadIdx.x == 0) *p.t = t + 1;
    }
}

template <int P, bool LOCAL>
cudaError_t launch_sw(const StepParams &p, int mode, cudaStream_t st) {
    static int per_sm = -1, sms = 0;
    if (per_sm < 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solids_step<P, LOCAL>,
                                                              SW_BLOCK, 0);
        if (e != cudaSuccess) return e;
    }
    const int work = p.nsolid > p.nmoving ? p.nsolid : p.nmoving;
    int blocks = (work + WARPS - 1) / WARPS;
    const int cap = per_sm * sms;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    StepParams pp = p;
    int m = mode;
    void *args[] = {&pp, &m};
    return cudaLaunchCooperativeKernel((const void *)k_solids_step<P, LOCAL>, dim3(blocks),
                                       dim3(SW_BLOCK), args, 0, st);
}

}  // namespace

cudaError_t launch_solids(const StepParams &p, int mode, cudaStream_t st) {
    if (p.nsolid == 0) return cudaSuccess;
    const bool local = p.rho_w_mode == LBM_RHOW_LOCAL;
    switch (p.precision) {
        case LBM_FP64: return local ? launch_sw<LBM_FP64, true>(p, mode, st)
                                    : launch_sw<LBM_FP64, false>(p, mode, st);
        case LBM_FP32_DEV: return local ? launch_sw<LBM_FP32_DEV, true>(p, mode, st)
                                        : launch_sw<LBM_FP32_DEV, false>(p, mode, st);
        default: return local ? launch_sw<LBM_FP16_DEV, true>(p, mode, st)
                              : launch_sw<LBM_FP16_DEV, false>(p, mode, st);
    }
}

}  // namespace gbm
