// Fused pull-advection + half-way bounce-back + BGK collision (Eq. 1-3, Eq. 8).
//
// One thread per node, x fastest, so every population plane is read and
// written with consecutive addresses across a warp.  The nine pulls are issued
// unconditionally (a bounced direction loads a neighbour that is later
// discarded, which costs no extra DRAM traffic because that row is streamed
// anyway); nodes next to a solid or a wall then take the rare path that
// replaces the bounced populations by f~_opp(x) + 6 w_i rho_w (e_i . v).
//
// Storage: FP64 stores f_i; the deviation modes store f_i - w_i (FP32 or
// FP16) and compute in FP32 entirely in deviation form, so that the small
// deviations keep their relative precision:
//   drho = sum d_i,  rho = 1 + drho,  rho u = sum e_i d_i,
//   deq_i = w_i (drho + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u.u)).
#include "lbm_internal.cuh"

namespace gbm {

namespace {

// Velocity of the wall or solid the population arriving at (x, y) along e_i
// was bounced from (its source x - e_i is solid or outside the domain).
__device__ __forceinline__ void source_velocity(const StepParams &p, int x, int y, int i,
                                                double &vx, double &vy) {
    const Lattice &L = p.L;
    int sx = x - cx(i), sy = y - cy(i);
    vx = 0.0;
    vy = 0.0;
    if (L.bc_y == LBM_WALL && (sy < 0 || sy >= L.ny)) {
        vx = sy < 0 ? p.wall_ux0 : p.wall_ux1;  // channel walls move along x
        return;
    }
    int xs, ys;
    if (!locate(L, sx, sy, xs, ys)) return;  // resting wall (or open column) in x
    uint16_t s = p.owner[cell_of(L, xs, ys)];
    if (s == FLUID) return;
    const DSolid &b = p.S[s];
    double dx, dy;
    // boundary point halfway between x and x - e_i
    point_velocity(L, b.x, b.y, b.vx, b.vy, b.om, (double)x - 0.5 * cx(i),
                   (double)y - 0.5 * cy(i), vx, vy, dx, dy);
}

// Post-collision populations (storage convention) of node (x, y).
template <int P, bool FORCE, bool LOCAL>
__device__ __forceinline__ void update_node(const StepParams &p,
                                            const typename Prec<P>::S *__restrict__ fin, int x,
                                            int y, uint16_t fl, typename Prec<P>::C (&out)[9]) {
    using C = typename Prec<P>::C;
    const Lattice &L = p.L;
    const long long k = cell_of(L, x, y);
    const bool per_x = L.bc_x == LBM_PERIODIC, per_y = L.bc_y == LBM_PERIODIC;
    C g[9];
#pragma unroll
    for (int i = 0; i < 9; i++) {
        int xs = x - cx(i), ys = y - cy(i);
        // wrap along periodic axes; clamp elsewhere (the value is then bounced)
        if (xs < 0) xs = per_x ? xs + L.nx : 0;
        if (xs >= L.nx) xs = per_x ? xs - L.nx : L.nx - 1;
        if (ys < 0) ys = per_y ? ys + L.ny : 0;
        if (ys >= L.ny) ys = per_y ? ys - L.ny : L.ny - 1;
        g[i] = ld(fin + (long long)i * L.plane + cell_of(L, xs, ys));
    }
    if (fl & 0x1FEu) {
        // half-way bounce-back with the moving-wall term
        C rho_w = (C)p.rho0;
        if (LOCAL) {
            C s = 0;
#pragma unroll
            for (int j = 0; j < 9; j++) s += ld(fin + (long long)j * L.plane + k);
            rho_w = Prec<P>::dev ? (C)1 + s : s;
        }
#pragma unroll
        for (int i = 1; i < 9; i++) {
            if (!((fl >> i) & 1u)) continue;
            double vx, vy;
            source_velocity(p, x, y, i, vx, vy);
            C back = ld(fin + (long long)opp(i) * L.plane + k);
            C ev = (C)(cx(i) * vx + cy(i) * vy);
            g[i] = back + (C)6 * wgt<C>(i) * rho_w * ev;
        }
    }
    C s0 = 0, jx = 0, jy = 0;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        s0 += g[i];
        jx += (C)cx(i) * g[i];
        jy += (C)cy(i) * g[i];
    }
    const C rho = Prec<P>::dev ? (C)1 + s0 : s0;
    const C Fx = (C)p.body_x, Fy = (C)p.body_y;
    const C inv = (C)1 / rho;
    const C ux = FORCE ? (jx + (C)0.5 * Fx) * inv : jx * inv;
    const C uy = FORCE ? (jy + (C)0.5 * Fy) * inv : jy * inv;
    const C uu = ux * ux + uy * uy;
    const C om = (C)p.omega;
    if (!(rho > (C)0) || !(fabs((double)ux) < 1e30) || !(fabs((double)uy) < 1e30))
        atomicOr(p.status, 1);
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const C eu = (C)cx(i) * ux + (C)cy(i) * uy;
        const C poly = (C)3 * eu + (C)4.5 * eu * eu - (C)1.5 * uu;
        C eq;
        if (Prec<P>::dev) eq = wgt<C>(i) * (s0 + rho * poly);  // f_eq - w_i
        else eq = rho * wgt<C>(i) * ((C)1 + poly);
        C o = g[i] - (g[i] - eq) * om;
        if (FORCE) {
            o += ((C)1 - (C)0.5 * om) * wgt<C>(i) *
                 ((C)3 * (((C)cx(i) - ux) * Fx + ((C)cy(i) - uy) * Fy) +
                  (C)9 * eu * ((C)cx(i) * Fx + (C)cy(i) * Fy));
        }
        out[i] = o;
    }
}

template <int P, bool FORCE, bool LOCAL>
__global__ void __launch_bounds__(SC_BLOCK_X) k_stream_collide(const StepParams p) {
    using S = typename Prec<P>::S;
    using C = typename Prec<P>::C;
    const Lattice &L = p.L;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= L.nx) return;
    const long long t = *p.t;
    const S *__restrict__ fin = static_cast<const S *>((t & 1) ? p.f1 : p.f0);
    S *__restrict__ fout = static_cast<S *>((t & 1) ? p.f0 : p.f1);
    const long long k = cell_of(L, x, y);
    const uint16_t fl = p.flags[k];
    if (fl & 1u) return;  // solid node: no populations
    C out[9];
    if (L.bc_x == LBM_OPEN && x == 0) {
        // equilibrium inlet with the parabolic profile
        const double h = (double)L.ny, yy = (double)y + 0.5;
        const C u = (C)(4.0 * p.umax * yy * (h - yy) / (h * h));
        const C r = (C)p.rho0;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const C eu = (C)cx(i) * u;
            const C poly = (C)3 * eu + (C)4.5 * eu * eu - (C)1.5 * u * u;
            out[i] = Prec<P>::dev ? wgt<C>(i) * ((r - (C)1) + r * poly)
                                  : r * wgt<C>(i) * ((C)1 + poly);
        }
    } else if (L.bc_x == LBM_OPEN && x == L.nx - 1 && !(p.flags[k - 1] & 1u)) {
        // outlet: copy of the updated column nx - 2
        update_node<P, FORCE, LOCAL>(p, fin, x - 1, y, p.flags[k - 1], out);
    } else {
        update_node<P, FORCE, LOCAL>(p, fin, x, y, fl, out);
    }
#pragma unroll
    for (int i = 0; i < 9; i++) st(fout + (long long)i * L.plane + k, out[i]);
}

template <int P, bool FORCE, bool LOCAL>
cudaError_t launch_sc(const StepParams &p, cudaStream_t st) {
    dim3 grid((p.L.nx + SC_BLOCK_X - 1) / SC_BLOCK_X, p.L.ny);
    k_stream_collide<P, FORCE, LOCAL><<<grid, SC_BLOCK_X, 0, st>>>(p);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_sc_p(const StepParams &p, cudaStream_t st) {
    const bool force = p.body_x != 0.0 || p.body_y != 0.0;
    const bool local = p.rho_w_mode == LBM_RHOW_LOCAL;
    if (force) return local ? launch_sc<P, true, true>(p, st) : launch_sc<P, true, false>(p, st);
    return local ? launch_sc<P, false, true>(p, st) : launch_sc<P, false, false>(p, st);
}

}  // namespace

cudaError_t launch_stream_collide(const StepParams &p, cudaStream_t st) {
    switch (p.precision) {
        case LBM_FP64: return launch_sc_p<LBM_FP64>(p, st);
        case LBM_FP32_DEV: return launch_sc_p<LBM_FP32_DEV>(p, st);
        default: return launch_sc_p<LBM_FP16_DEV>(p, st);
    }
}

}  // namespace gbm
