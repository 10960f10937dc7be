// Device code of the fused pull-advection + half-way bounce-back + BGK
// collision (Eq. 1-3, Eq. 8), shared by the single-domain kernel
// (k_stream_collide.cu) and the batch kernels (k_stream_collide_batch.cu).
// Each translation unit compiles its own copy, so that the register budget of
// one kernel family does not constrain the other's per-node path.
//
// Layout: SoA planes f_i[ny][pitch], x fastest, pitch a multiple of 64.
// Every thread owns V consecutive nodes of one row, V chosen so that one
// population of those nodes is 16 bytes (FP64: 2, FP32: 4, FP16: 8).  Each of
// the nine pulls is one aligned 128-bit load from the source row (y - c_y);
// the x-shifted pulls (c_x = +-1) take the missing neighbour element from the
// adjacent lane with a warp shuffle (lanes 0 and 31 load it directly, wrapped
// at the row ends), so DRAM sees each population plane read once, fully
// coalesced.  Results go out as nine 128-bit stores (nodes in the row padding
// store zeros).  Nodes next to a solid or a wall and the first and last
// column take a per-node path, which in the batch kernels (OPEN) also
// computes the columns of an open channel; the single-domain kernel leaves
// those to a separate pass (open_row), to keep its per-node path small.
//
// Bounce-back: a node whose flags word has bit i set (x - e_i solid or
// outside) replaces population i by f~_opp(x) + 6 w_i rho_w (e_i . v), v the
// velocity of the wall or solid at x - e_i / 2.  Solid nodes store zeros.
//
// Storage: FP64 stores f_i; the deviation modes store f_i - w_i (FP32 or
// FP16) and compute in FP32 entirely in deviation form, so that the small
// deviations keep their relative precision:
//   drho = sum d_i,  rho = 1 + drho,  rho u = sum e_i d_i,
//   deq_i = w_i (drho + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u.u)).
#pragma once
#include "lbm_internal.cuh"

namespace gbm {

namespace {

template <int P> struct Raw;
template <> struct Raw<LBM_FP64> { using R = double; };
template <> struct Raw<LBM_FP32_DEV> { using R = float; };
template <> struct Raw<LBM_FP16_DEV> { using R = unsigned short; };

template <int BYTES> struct Word;
template <> struct Word<2> { using T = uint16_t; };
template <> struct Word<4> { using T = uint32_t; };
template <> struct Word<8> { using T = uint2; };
template <> struct Word<16> { using T = uint4; };

// V consecutive values of one population plane, loaded as one word
template <class R, int V> union Pack {
    typename Word<sizeof(R) * V>::T u;
    R r[V];
};
template <int V> union FlagPack {
    typename Word<2 * V>::T u;
    uint16_t f[V];
};

__device__ __forceinline__ double cvt(double v) { return v; }
__device__ __forceinline__ float cvt(float v) { return v; }
__device__ __forceinline__ float cvt(unsigned short v) { return __half2float(__ushort_as_half(v)); }
__device__ __forceinline__ void put(double &d, double v) { d = v; }
__device__ __forceinline__ void put(float &d, float v) { d = v; }
__device__ __forceinline__ void put(unsigned short &d, float v) {
    d = __half_as_ushort(__float2half_rn(v));
}

// two adjacent values of a population plane at once (FP16: one half2)
__device__ __forceinline__ void put2(float *d, float a, float b) {
    d[0] = a;
    d[1] = b;
}
__device__ __forceinline__ void put2(unsigned short *d, float a, float b) {
    *reinterpret_cast<__half2 *>(d) = __floats2half2_rn(a, b);
}

// Paired FP32 arithmetic: one instruction for the same operation on two nodes.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ unsigned short shfl_up1(unsigned short v) {
    return (unsigned short)__shfl_up_sync(0xffffffffu, (int)v, 1);
}
__device__ __forceinline__ double shfl_dn1(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ unsigned short shfl_dn1(unsigned short v) {
    return (unsigned short)__shfl_down_sync(0xffffffffu, (int)v, 1);
}

// Replace the bounced populations of node (x, y) (rare path): population i,
// whose source x - e_i is a wall or a solid, becomes f~_opp(x) + 6 w_i rho_w
// (e_i . v) with v the wall's or solid's velocity at x - e_i / 2 (Sec. III.A;
// the moving-wall term).
// BND: disks with the interpolated boundary (LBM_INTERPOLATED), compiled only
// into the kernels that run the per-node path outside the vector path.
template <int P, bool LOCAL, bool BND = false>
__device__ __forceinline__ void bounce(const StepParams &p, const typename Raw<P>::R *fin, int x,
                                       int y, uint16_t fl, typename Prec<P>::C (&g)[9]) {
    using C = typename Prec<P>::C;
    const Lattice &L = p.L;
    const int k = y * L.pitch + x;
    const int plane = (int)L.plane;
    C rho_w = pick<C>(p.rho0, p.rho0_f);
    if (LOCAL) {
        C s = 0;
#pragma unroll
        for (int j = 0; j < 9; j++) s += cvt(fin[j * plane + k]);
        rho_w = Prec<P>::dev ? (C)1 + s : s;
    }
#pragma unroll
    for (int i = 1; i < 9; i++) {
        if (!((fl >> i) & 1u)) continue;
        const int sx = x - cx(i), sy = y - cy(i);
        C vx = 0, vy = 0;
        int xs, ys;
        if (L.bc_y == LBM_WALL && (sy < 0 || sy >= L.ny)) {
            vx = sy < 0 ? pick<C>(p.wall_ux0, p.wall_ux0_f) : pick<C>(p.wall_ux1, p.wall_ux1_f);
        } else if (locate(L, sx, sy, xs, ys)) {
            const uint16_t o = p.owner[cell_of(L, xs, ys)];
            if (BND && o != FLUID) {
                // the cut at fraction q of the link towards the wall; linear
                // interpolation of the returned population (deviation form
                // as well: the weights sum to one):
                //   q < 1/2:  2q f~_opp(x) + (1 - 2q) f~_opp(x + e_i) + M
                //   q >= 1/2: (f~_opp(x) + M) / (2q) + (2q - 1) / (2q) f~_i(x)
                // M = 6 w_i rho_w (e_i . v), v at the cut x - q e_i; half-way
                // value where x + e_i is not a fluid node
                const DSolid &b = p.S[o];
                C q, ux, uy;
                if (Prec<P>::dev) {
                    // FP32: the offset from the centre's nearest image, split
                    int di = x - b.xwi, dj = y - b.ywi;
                    if (L.bc_x == LBM_PERIODIC) {
                        if (2 * di > L.nx) di -= L.nx;
                        else if (2 * di < -L.nx) di += L.nx;
                    }
                    if (L.bc_y == LBM_PERIODIC) {
                        if (2 * dj > L.ny) dj -= L.ny;
                        else if (2 * dj < -L.ny) dj += L.ny;
                    }
                    q = (C)link_fraction_split(di, dj, b.xwr, b.ywr, b.r, -cx(i), -cy(i));
                    const C ddx = ((C)di - (C)b.xwr) - q * (C)cx(i);
                    const C ddy = ((C)dj - (C)b.ywr) - q * (C)cy(i);
                    ux = (C)b.vxf - (C)b.omf * ddy;
                    uy = (C)b.vyf + (C)b.omf * ddx;
                } else {
                    const double qd = link_fraction(L, b, x, y, opp(i));
                    double vxd, vyd, ddx, ddy;
                    point_velocity(L, b.x, b.y, b.vx, b.vy, b.om, (double)x - qd * cx(i),
                                   (double)y - qd * cy(i), vxd, vyd, ddx, ddy);
                    q = (C)qd;
                    ux = (C)vxd;
                    uy = (C)vyd;
                }
                const C m = (C)6 * wgt<C>(i) * rho_w * ((C)cx(i) * ux + (C)cy(i) * uy);
                const C back = cvt(fin[opp(i) * plane + k]);
                const C q2 = (C)2 * q;
                if (q2 >= (C)1) {
                    g[i] = (back + m) / q2 + ((q2 - (C)1) / q2) * cvt(fin[i * plane + k]);
                } else if (!((fl >> opp(i)) & 1u)) {
                    int xn, yn;
                    locate(L, x + cx(i), y + cy(i), xn, yn);
                    g[i] = q2 * back +
                           ((C)1 - q2) * cvt(fin[opp(i) * plane + yn * L.pitch + xn]) + m;
                } else {
                    g[i] = back + m;
                }
                continue;
            }
            if (o != FLUID) {
                const DSolid &b = p.S[o];
                vx = pick<C>(b.vx, b.vxf);
                vy = pick<C>(b.vy, b.vyf);
                if (b.omf != 0.0f) {
                    // x - e_i / 2 relative to R, nearest periodic image
                    C dx, dy;
                    if (Prec<P>::dev) {
                        dx = (C)(x - b.xwi) - (C)(0.5f * cx(i)) - (C)b.xwr;
                        dy = (C)(y - b.ywi) - (C)(0.5f * cy(i)) - (C)b.ywr;
                    } else {
                        dx = (C)((double)x - 0.5 * cx(i) - b.xw);
                        dy = (C)((double)y - 0.5 * cy(i) - b.yw);
                    }
                    if (L.bc_x == LBM_PERIODIC) {
                        if (dx > (C)(0.5 * L.nx)) dx -= (C)L.nx;
                        else if (dx < (C)(-0.5 * L.nx)) dx += (C)L.nx;
                    }
                    if (L.bc_y == LBM_PERIODIC) {
                        if (dy > (C)(0.5 * L.ny)) dy -= (C)L.ny;
                        else if (dy < (C)(-0.5 * L.ny)) dy += (C)L.ny;
                    }
                    const C om = pick<C>(b.om, b.omf);
                    vx -= om * dy;
                    vy += om * dx;
                }
            }
        }
        const C back = cvt(fin[opp(i) * plane + k]);
        g[i] = back + (C)6 * wgt<C>(i) * rho_w * ((C)cx(i) * vx + (C)cy(i) * vy);
    }
}

// BGK collision (with Guo forcing when FORCE) of one node in place.
template <int P, bool FORCE>
__device__ __forceinline__ void collide(const StepParams &p, typename Prec<P>::C (&g)[9]) {
    using C = typename Prec<P>::C;
    C s0 = 0, jx = 0, jy = 0;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        s0 += g[i];
        jx += (C)cx(i) * g[i];
        jy += (C)cy(i) * g[i];
    }
    const C rho = Prec<P>::dev ? (C)1 + s0 : s0;
    const C Fx = pick<C>(p.body_x, p.body_xf), Fy = pick<C>(p.body_y, p.body_yf);
    const C inv = (C)1 / rho;
    const C ux = FORCE ? (jx + (C)0.5 * Fx) * inv : jx * inv;
    const C uy = FORCE ? (jy + (C)0.5 * Fy) * inv : jy * inv;
    const C uu = ux * ux + uy * uy;
    const C om = pick<C>(p.omega, p.omega_f);
    if (!(rho > (C)0) || !(fabs(ux) < (C)1e30) || !(fabs(uy) < (C)1e30)) atomicOr(p.status, 1);
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
        g[i] = o;
    }
}

// MRT collision of one node in place (Sec. IV names the model and its rates
// S = diag(0, 1.64, 1.54, 0, 1.9, 0, 1.9, 1/tau, 1/tau)): the moments of the
// basis (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy) relax towards those of
// the Eq. 8 equilibrium, -2 rho + 3 j^2 / rho, rho - 3 j^2 / rho, -j,
// (j_x^2 - j_y^2) / rho and j_x j_y / rho (in the deviation modes minus the
// moments of the weights, which are 1, -2, 1 and zeros), and the change goes
// back to the populations through the transposed basis over the squared row
// norms (36, 36, 12, 12, 4, 4).  No body force.  CHECK: flag a non-physical
// state (the vector path checks its fluid nodes itself; solid nodes there
// hold no state).
template <int P, bool CHECK>
__device__ __forceinline__ void collide_mrt(const StepParams &p, typename Prec<P>::C (&g)[9]) {
    using C = typename Prec<P>::C;
    const C ax = g[1] + g[2] + g[3] + g[4], dg = g[5] + g[6] + g[7] + g[8];
    const C s0 = g[0] + ax + dg;
    const C jx = g[1] - g[3] + g[5] - g[6] - g[7] + g[8];
    const C jy = g[2] - g[4] + g[5] + g[6] - g[7] - g[8];
    const C rho = Prec<P>::dev ? (C)1 + s0 : s0;
    const C inv = (C)1 / rho;
    if (CHECK && (!(rho > (C)0) || !(fabs(jx * inv) < (C)1e30) || !(fabs(jy * inv) < (C)1e30)))
        atomicOr(p.status, 1);
    const C jj = (jx * jx + jy * jy) * inv;
    const C e = (C)-4 * g[0] - ax + (C)2 * dg;
    const C eps = (C)4 * g[0] - (C)2 * ax + dg;
    const C qx = (C)2 * (g[3] - g[1]) + g[5] - g[6] - g[7] + g[8];
    const C qy = (C)2 * (g[4] - g[2]) + g[5] + g[6] - g[7] - g[8];
    const C pxx = g[1] - g[2] + g[3] - g[4];
    const C pxy = g[5] - g[6] + g[7] - g[8];
    const C eeq = Prec<P>::dev ? (C)-2 * s0 + (C)3 * jj : (C)-2 * rho + (C)3 * jj;
    const C epseq = Prec<P>::dev ? s0 - (C)3 * jj : rho - (C)3 * jj;
    const C om = pick<C>(p.omega, p.omega_f);
    const C de = (C)(1.64 / 36.0) * (e - eeq);
    const C dp = (C)(1.54 / 36.0) * (eps - epseq);
    const C dqx = (C)(1.9 / 12.0) * (qx + jx);
    const C dqy = (C)(1.9 / 12.0) * (qy + jy);
    const C dxx = (C)0.25 * om * (pxx - (jx * jx - jy * jy) * inv);
    const C dxy = (C)0.25 * om * (pxy - jx * jy * inv);
    const C a = -de - (C)2 * dp, b = (C)2 * de + dp;
    g[0] -= (C)4 * (dp - de);
    g[1] -= a - (C)2 * dqx + dxx;
    g[2] -= a - (C)2 * dqy - dxx;
    g[3] -= a + (C)2 * dqx + dxx;
    g[4] -= a + (C)2 * dqy - dxx;
    g[5] -= b + dqx + dqy + dxy;
    g[6] -= b - dqx + dqy - dxy;
    g[7] -= b - dqx - dqy + dxy;
    g[8] -= b + dqx - dqy - dxy;
}

// Inlet profile of an open channel at row y: u_in = 4 umax y' (ny - y') / ny^2,
// y' = y + 1/2 (walls at y = -1/2 and ny - 1/2); in the precision C of the
// kernel (no FP64 arithmetic in the FP32 kernels).
template <class C>
__device__ __forceinline__ C inlet_ux(const StepParams &p, int y) {
    const C h = (C)p.L.ny, yy = (C)y + (C)0.5;
    return (C)4 * pick<C>(p.umax, p.umax_f) * yy * (h - yy) / (h * h);
}

// feq(rho0, (u_in, 0)) into g (deviation form in the deviation modes).
template <int P>
__device__ __forceinline__ void inlet_equilibrium(const StepParams &p, typename Prec<P>::C u_in,
                                                  typename Prec<P>::C (&g)[9]) {
    using C = typename Prec<P>::C;
    const C r = pick<C>(p.rho0, p.rho0_f);
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const C eu = (C)cx(i) * u_in;
        const C poly = (C)3 * eu + (C)4.5 * eu * eu - (C)1.5 * u_in * u_in;
        g[i] = Prec<P>::dev ? wgt<C>(i) * ((r - (C)1) + r * poly) : r * wgt<C>(i) * ((C)1 + poly);
    }
}

// Non-equilibrium extrapolation onto an open column from the post-collision
// populations g of its inner neighbour n, in place: g + feq(rho_b, u_b) -
// feq(rho_n, u_n), with rho_n, u_n the neighbour's density and velocity (BGK
// keeps rho and rho u; Guo forcing adds F to rho u).  Inlet: u_b = (u_in, 0),
// rho_b = rho_n; outlet: rho_b = rho0, u_b = u_n.
template <int P, bool FORCE>
__device__ __forceinline__ void extrapolate_open(const StepParams &p, bool inlet,
                                                 typename Prec<P>::C u_in,
                                                 typename Prec<P>::C (&g)[9]) {
    using C = typename Prec<P>::C;
    C s0 = 0, jx = 0, jy = 0;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        s0 += g[i];
        jx += (C)cx(i) * g[i];
        jy += (C)cy(i) * g[i];
    }
    const C rn = Prec<P>::dev ? (C)1 + s0 : s0;
    if (FORCE) {
        jx -= (C)0.5 * pick<C>(p.body_x, p.body_xf);
        jy -= (C)0.5 * pick<C>(p.body_y, p.body_yf);
    }
    const C uxn = jx / rn, uyn = jy / rn;
    const C ub = inlet ? u_in : uxn, vb = inlet ? (C)0 : uyn;
    const C rb = inlet ? rn : pick<C>(p.rho0, p.rho0_f);
    const C uun = uxn * uxn + uyn * uyn, uub = ub * ub + vb * vb;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        const C en = (C)cx(i) * uxn + (C)cy(i) * uyn, eb = (C)cx(i) * ub + (C)cy(i) * vb;
        const C pn = (C)3 * en + (C)4.5 * en * en - (C)1.5 * uun;
        const C pb = (C)3 * eb + (C)4.5 * eb * eb - (C)1.5 * uub;
        g[i] += wgt<C>(i) * ((rb - rn) + rb * pb - rn * pn);
    }
}

// Complete update of one node, with periodic wrap, bounce-back and walls
// (beyond a non-periodic edge: a resting wall): used for the nodes the vector
// path leaves out (fluid nodes next to a solid or wall, the first and last
// column).  With OPEN, the columns of an open channel are computed here too:
// the update of the inner neighbour (x = 1 or nx - 2, recomputed from fin)
// followed by the non-equilibrium extrapolation; next to a solid neighbour
// the inlet is feq(rho0, u_in) and the outlet updates as a walled node.
// Without OPEN they update as walled nodes and a later pass (open_col)
// replaces them.
template <int P, bool FORCE, bool LOCAL, bool OPEN, int COLL = 0, bool BND = false>
__device__ __noinline__ void update_node(const StepParams &p, const typename Raw<P>::R *fin,
                                         typename Raw<P>::R *fout, int x, int y) {
    using C = typename Prec<P>::C;
    using R = typename Raw<P>::R;
    const Lattice &L = p.L;
    const int plane = (int)L.plane;
    const int k = y * L.pitch + x;
    const uint16_t fl = p.flags[k];
    C g[9];
    if (fl & 1u) {
#pragma unroll
        for (int i = 0; i < 9; i++) put(fout[i * plane + k], (C)0);
        return;
    }
    int xu = x;  // node whose update is computed
    uint16_t flu = fl;
    bool open = false;
    C u_in = 0;
    if (OPEN && L.bc_x == LBM_OPEN && (x == 0 || x == L.nx - 1)) {
        const uint16_t fln = p.flags[x == 0 ? k + 1 : k - 1];
        if (x == 0) u_in = inlet_ux<C>(p, y);
        if (!(fln & 1u)) {
            open = true;
            xu = x == 0 ? 1 : x - 1;
            flu = fln;
        } else if (x == 0) {
            inlet_equilibrium<P>(p, u_in, g);
#pragma unroll
            for (int i = 0; i < 9; i++) put(fout[i * plane + k], g[i]);
            return;
        }
    }
    const bool per_x = L.bc_x == LBM_PERIODIC, per_y = L.bc_y == LBM_PERIODIC;
#pragma unroll
    for (int i = 0; i < 9; i++) {
        int xs = xu - cx(i), ys = y - cy(i);
        // wrap along periodic axes; clamp elsewhere (the value is then bounced)
        if (xs < 0) xs = per_x ? xs + L.nx : 0;
        if (xs >= L.nx) xs = per_x ? xs - L.nx : L.nx - 1;
        if (ys < 0) ys = per_y ? ys + L.ny : 0;
        if (ys >= L.ny) ys = per_y ? ys - L.ny : L.ny - 1;
        g[i] = cvt(fin[i * plane + ys * L.pitch + xs]);
    }
    if (flu & 0x1FEu) bounce<P, LOCAL, BND>(p, fin, xu, y, flu, g);
    if constexpr (COLL == 1) collide_mrt<P, true>(p, g);
    else collide<P, FORCE>(p, g);
    if (OPEN && open) extrapolate_open<P, FORCE>(p, x == 0, u_in, g);
#pragma unroll
    for (int i = 0; i < 9; i++) {
        R v;
        put(v, g[i]);
        fout[i * plane + k] = v;
    }
}

// One tile: row y, nodes bx * SC_BLOCK_X * V .. + SC_BLOCK_X * V - 1 (the
// whole block works on the same tile).
// WALLS: bounce-back from the y walls on the vector path (FP32 and FP64 with
// rho_w = rho0 only; FP16 storage would round the bounced values).
template <int P, bool LOCAL>
__host__ __device__ constexpr bool walls_on_vector_path() { return !LOCAL && P != LBM_FP16_DEV; }

// DEFER: the per-node path is left to a later pass over the nodes next to
// solids and edges (the single-domain kernel); otherwise each thread runs it
// for its own nodes at the end of the tile.
// COLL: 0 = BGK, 1 = MRT (no body force, slow nodes inline).
template <int P, int V, bool FORCE, bool LOCAL, bool OPEN, bool WALLS = false, bool DEFER = false,
          int COLL = 0, bool BND = false>
__device__ __forceinline__ void sc_tile(const StepParams &p, int bx, int y) {
    static_assert(!WALLS || walls_on_vector_path<P, LOCAL>(), "wall rows need rho0 and R == C");
    using R = typename Raw<P>::R;
    using C = typename Prec<P>::C;
    const Lattice &L = p.L;
    const int lane = threadIdx.x & 31;
    const int x0 = (bx * SC_BLOCK_X + threadIdx.x) * V;
    // OPEN marks the batch kernels, whose case parameters keep the current
    // populations in f0 and the next in f1 (swapped as the clock advances);
    // a single domain selects by the parity of its step counter
    const long long t = OPEN ? 0 : *p.t;
    const R *__restrict__ fin = static_cast<const R *>((t & 1) ? p.f1 : p.f0);
    R *__restrict__ fout = static_cast<R *>((t & 1) ? p.f0 : p.f1);
    const int plane = (int)L.plane;
    const int xl = min(x0, L.pitch - V);  // in-bounds load position for every lane
    int ym = y - 1, yp = y + 1;
    if (ym < 0) ym = L.bc_y == LBM_PERIODIC ? L.ny - 1 : 0;
    if (yp >= L.ny) yp = L.bc_y == LBM_PERIODIC ? 0 : L.ny - 1;
    const int rm = ym * L.pitch, r0 = y * L.pitch, rp = yp * L.pitch;
#define SROW(i) (cy(i) == 1 ? rm : (cy(i) == -1 ? rp : r0))

    Pack<R, V> raw[9];
#pragma unroll
    for (int i = 0; i < 9; i++)
        raw[i].u = __ldg(reinterpret_cast<const typename Word<sizeof(R) * V>::T *>(
            fin + i * plane + SROW(i) + xl));
    FlagPack<V> fl;
    fl.u = *reinterpret_cast<const typename Word<2 * V>::T *>(p.flags + r0 + xl);
    // neighbour elements of the x-shifted pulls at the warp's ends; at the
    // row ends they are wrong, but those columns take the per-node path
    R hl[3] = {R(0), R(0), R(0)};
    if (lane == 0) {
        const int xh = max(x0 - 1, 0);
        hl[0] = fin[1 * plane + SROW(1) + xh];
        hl[1] = fin[5 * plane + SROW(5) + xh];
        hl[2] = fin[8 * plane + SROW(8) + xh];
    } else if (lane == 31) {
        const int xh = min(x0 + V, L.pitch - 1);
        hl[0] = fin[3 * plane + SROW(3) + xh];
        hl[1] = fin[6 * plane + SROW(6) + xh];
        hl[2] = fin[7 * plane + SROW(7) + xh];
    }
    R halo[9];
#pragma unroll
    for (int i = 0; i < 9; i++) {
        halo[i] = R(0);
        if (cx(i) == 1) halo[i] = shfl_up1(raw[i].r[V - 1]);
        else if (cx(i) == -1) halo[i] = shfl_dn1(raw[i].r[0]);
    }
#undef SROW
    if (x0 >= L.nx) return;
    if (lane == 0) {
        halo[1] = hl[0];
        halo[5] = hl[1];
        halo[8] = hl[2];
    } else if (lane == 31) {
        halo[3] = hl[0];
        halo[6] = hl[1];
        halo[7] = hl[2];
    }
    // Wall rows (WALLS): the populations that arrive from the wall (y = -1/2
    // or ny - 1/2) are the node's own opposite populations plus the moving-wall
    // term, 6 w_i rho0 (e_i . u_wall) (Sec. III.A, rho_w = rho0).  They are
    // written where the pulls below read them, so the row stays on the vector
    // path; nodes with any other bounced population still take the per-node path.
    uint16_t wall_bits = 0;
    if (WALLS && L.bc_y == LBM_WALL && (y == 0 || y == L.ny - 1)) {
        const bool lo = y == 0;
        wall_bits = lo ? 0x64 : 0x190;  // {2, 5, 6} at y = 0, {4, 7, 8} at y = ny - 1
        const C uw = lo ? pick<C>(p.wall_ux0, p.wall_ux0_f) : pick<C>(p.wall_ux1, p.wall_ux1_f);
        const C rho_w = pick<C>(p.rho0, p.rho0_f);
#pragma unroll
        for (int i = 1; i < 9; i++) {
            if (!((wall_bits >> i) & 1u)) continue;
            Pack<R, V> own;  // the node's own population opp(i), row y
            own.u = __ldg(reinterpret_cast<const typename Word<sizeof(R) * V>::T *>(
                fin + opp(i) * plane + r0 + xl));
            const C term = (C)6 * wgt<C>(i) * rho_w * ((C)cx(i) * uw);
#pragma unroll
            for (int j = 0; j < V; j++) {
                const R b = (R)(cvt(own.r[j]) + term);
                if (cx(i) == 0) raw[i].r[j] = b;
                else if (cx(i) == 1) {
                    if (j == 0) halo[i] = b;
                    else raw[i].r[j - 1] = b;
                } else {
                    if (j == V - 1) halo[i] = b;
                    else raw[i].r[j + 1] = b;
                }
            }
        }
    }
#define PULL(i, j) \
    cvt(cx(i) == 0 ? raw[i].r[j] \
                   : (cx(i) == 1 ? ((j) == 0 ? halo[i] : raw[i].r[(j) - 1]) \
                                 : ((j) == V - 1 ? halo[i] : raw[i].r[(j) + 1])))
    uint32_t slow = 0;  // bit j: node j needs the per-node path
    // node j needs the per-node path, or has a non-physical state (flagged)
    auto classify = [&](int j, C r, C vx, C vy) {
        const uint16_t f = fl.f[j];
        const int x = x0 + j;
        if (!(f & 1u) && ((f & 0x1FEu & ~wall_bits) || x == 0 || x == L.nx - 1)) slow |= 1u << j;
        else if (!(f & 1u) && x < L.nx &&
                 (!(r > (C)0) || !(fabs(vx) < (C)1e30) || !(fabs(vy) < (C)1e30)))
            atomicOr(p.status, 1);
    };
    if constexpr (COLL == 1) {
        // MRT, one node at a time
        static_assert(!FORCE && !DEFER, "MRT runs without body force and with inline slow nodes");
        Pack<R, V> o[9];
#pragma unroll
        for (int j = 0; j < V; j++) {
            C g[9];
            C a = 0, jx = 0, jy = 0;
#pragma unroll
            for (int i = 0; i < 9; i++) {
                g[i] = PULL(i, j);
                a += g[i];
                jx += (C)cx(i) * g[i];
                jy += (C)cy(i) * g[i];
            }
            const C r = Prec<P>::dev ? (C)1 + a : a;
            classify(j, r, jx / r, jy / r);
            collide_mrt<P, false>(p, g);
#pragma unroll
            for (int i = 0; i < 9; i++) put(o[i].r[j], (fl.f[j] & 1u) ? (C)0 : g[i]);
        }
#pragma unroll
        for (int i = 0; i < 9; i++)
            *reinterpret_cast<typename Word<sizeof(R) * V>::T *>(fout + i * plane + r0 + x0) = o[i].u;
    } else if constexpr (Prec<P>::dev && !FORCE && V % 2 == 0) {
        // Deviation form, two nodes per instruction (FADD2 / FMUL2 / FFMA2).
        // With E_i = s0 + rho (3 e_i.u + 4.5 (e_i.u)^2 - 1.5 u.u) the
        // equilibrium deviation is w_i E_i, and BGK gives
        // (1 - omega) g_i + omega w_i E_i.  Opposite populations share
        // A = s0 - 1.5 rho u.u and the even part 4.5 rho (e.u)^2; the odd part
        // 3 rho e.u changes sign.
        const float om = p.omega_f;
        const float2 omc = dup2(1.f - om);
        Pack<R, V> o[9];
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            float2 g[9];
#pragma unroll
            for (int i = 0; i < 9; i++) g[i] = make_float2(PULL(i, j), PULL(i, j + 1));
            const float2 s0 = add2(add2(add2(g[0], g[1]), add2(g[2], g[3])),
                                   add2(add2(g[4], g[5]), add2(add2(g[6], g[7]), g[8])));
            const float2 jx = sub2(add2(add2(g[1], g[5]), g[8]), add2(add2(g[3], g[6]), g[7]));
            const float2 jy = sub2(add2(add2(g[2], g[5]), g[6]), add2(add2(g[4], g[7]), g[8]));
            const float2 rho = add2(dup2(1.f), s0);
            const float2 inv = make_float2(1.f / rho.x, 1.f / rho.y);
            const float2 ux = mul2(jx, inv), uy = mul2(jy, inv);
            classify(j, rho.x, ux.x, uy.x);
            classify(j + 1, rho.y, ux.y, uy.y);
            const float2 A = fma2(mul2(dup2(-1.5f), rho), fma2(ux, ux, mul2(uy, uy)), s0);
            float2 out[9];
            out[0] = fma2(dup2(om * wgt<float>(0)), A, mul2(omc, g[0]));
            // (i, opp(i)) with e_i.u = eu: (1, 3) ux, (2, 4) uy, (5, 7) ux + uy, (6, 8) uy - ux
            auto pair = [&](int i, int k, float2 eu) {
                const float2 q = mul2(rho, eu);
                const float2 sym = fma2(q, mul2(dup2(4.5f), eu), A);
                const float2 ow = dup2(om * wgt<float>(i));
                out[i] = fma2(ow, fma2(dup2(3.f), q, sym), mul2(omc, g[i]));
                out[k] = fma2(ow, fma2(dup2(-3.f), q, sym), mul2(omc, g[k]));
            };
            pair(1, 3, ux);
            pair(2, 4, uy);
            pair(5, 7, add2(ux, uy));
            pair(6, 8, sub2(uy, ux));
            const bool s_a = fl.f[j] & 1u, s_b = fl.f[j + 1] & 1u;  // solid nodes store zeros
#pragma unroll
            for (int i = 0; i < 9; i++)
                put2(&o[i].r[j], s_a ? 0.f : out[i].x, s_b ? 0.f : out[i].y);
        }
#pragma unroll
        for (int i = 0; i < 9; i++)
            *reinterpret_cast<typename Word<sizeof(R) * V>::T *>(fout + i * plane + r0 + x0) = o[i].u;
    } else {
    // moments of every node from the pulled populations
    C s0[V], ux[V], uy[V], rho[V];
#pragma unroll
    for (int j = 0; j < V; j++) {
        C a = 0, jx = 0, jy = 0;
#pragma unroll
        for (int i = 0; i < 9; i++) {
            const C g = PULL(i, j);
            a += g;
            jx += (C)cx(i) * g;
            jy += (C)cy(i) * g;
        }
        const C r = Prec<P>::dev ? (C)1 + a : a;
        const C inv = (C)1 / r;
        s0[j] = a;
        rho[j] = r;
        ux[j] = FORCE ? (jx + (C)0.5 * pick<C>(p.body_x, p.body_xf)) * inv : jx * inv;
        uy[j] = FORCE ? (jy + (C)0.5 * pick<C>(p.body_y, p.body_yf)) * inv : jy * inv;
        classify(j, r, ux[j], uy[j]);
    }
    // relax towards equilibrium, one population plane at a time
    const C om = pick<C>(p.omega, p.omega_f);
#pragma unroll
    for (int i = 0; i < 9; i++) {
        Pack<R, V> o;
#pragma unroll
        for (int j = 0; j < V; j++) {
            const C g = PULL(i, j);
            const C eu = (C)cx(i) * ux[j] + (C)cy(i) * uy[j];
            const C uu = ux[j] * ux[j] + uy[j] * uy[j];
            const C poly = (C)3 * eu + (C)4.5 * eu * eu - (C)1.5 * uu;
            const C eq = Prec<P>::dev ? wgt<C>(i) * (s0[j] + rho[j] * poly)
                                      : rho[j] * wgt<C>(i) * ((C)1 + poly);
            C v = g - (g - eq) * om;
            if (FORCE) {
                const C Fx = pick<C>(p.body_x, p.body_xf), Fy = pick<C>(p.body_y, p.body_yf);
                v += ((C)1 - (C)0.5 * om) * wgt<C>(i) *
                     ((C)3 * (((C)cx(i) - ux[j]) * Fx + ((C)cy(i) - uy[j]) * Fy) +
                      (C)9 * eu * ((C)cx(i) * Fx + (C)cy(i) * Fy));
            }
            put(o.r[j], (fl.f[j] & 1u) ? (C)0 : v);  // solid nodes store zeros
        }
        *reinterpret_cast<typename Word<sizeof(R) * V>::T *>(fout + i * plane + r0 + x0) = o.u;
    }
    }
#undef PULL
    // nodes next to a solid or a wall and the first/last column
    if constexpr (!DEFER) {
        while (slow) {
            const int j = __ffs(slow) - 1;
            slow &= slow - 1;
            update_node<P, FORCE, LOCAL, OPEN, COLL, BND>(p, fin, fout, x0 + j, y);
        }
    }
}

// Open channel (bc_x = LBM_OPEN), after the fused kernel of step t has
// written the populations of t+1 into f: column x = 0 (inlet) or x = nx - 1
// (outlet) of row y takes the non-equilibrium extrapolation of its inner
// neighbour's post-collision populations (extrapolate_open); next to a solid
// neighbour the inlet takes feq(rho0, u_in) and the outlet keeps its own
// update (a resting wall beyond the edge).  open_row does both columns.
template <int P, bool FORCE>
__device__ __forceinline__ void open_col(const StepParams &p, typename Raw<P>::R *f, int y,
                                         bool inlet) {
    using C = typename Prec<P>::C;
    const Lattice &L = p.L;
    const int plane = (int)L.plane;
    const int x = inlet ? 0 : L.nx - 1;
    const int k = y * L.pitch + x, kn = inlet ? k + 1 : k - 1;
    if (p.flags[k] & 1u) return;
    const C u_in = inlet ? inlet_ux<C>(p, y) : (C)0;
    C g[9];
    if (p.flags[kn] & 1u) {
        if (!inlet) return;
        inlet_equilibrium<P>(p, u_in, g);
    } else {
#pragma unroll
        for (int i = 0; i < 9; i++) g[i] = cvt(f[i * plane + kn]);
        extrapolate_open<P, FORCE>(p, inlet, u_in, g);
    }
#pragma unroll
    for (int i = 0; i < 9; i++) put(f[i * plane + k], g[i]);
}

template <int P, bool FORCE>
__device__ __forceinline__ void open_row(const StepParams &p, typename Raw<P>::R *f, int y) {
    open_col<P, FORCE>(p, f, y, true);
    open_col<P, FORCE>(p, f, y, false);
}

}  // namespace

}  // namespace gbm
