// Per-solid work of one step t -> t+1, in three launches.
//
// k_forces, one block per solid, and then k_ring run beside the
// advection-collision kernel of the step: they read the populations of time
// t, the owner map and the node flags (which that kernel also only reads),
// and write nothing that it reads.
//   k_forces: the momentum booked by the node-type changes of the previous
//      step (the solid's segment of the event list), the link sums of Eq. 4
//      and Eq. 5 over every fluid-solid link of time t (Eq. 6 and Eq. 7) ->
//      the force record of t; the motion t -> t+1 (prescribed, or
//      Newton-Euler on the Eq. 5 force; Eq. 4 when the context selects it for
//      comparison); the largest displacement of any solid since the last
//      pair test.
//   k_ring, one warp per moving solid:
//   P  only when some solid may have come within reach of another one since
//      the last test: the solid's near list, the solids whose centres are
//      closer than r_s + r_q + NEAR_REACH + NEAR_MARGIN at t or t+1
//   R  on the ring (old disk XOR new disk): the owner at t and at t+1 from
//      the geometry of the solid and of its near list (lowest id where disks
//      overlap), so that no map of the old owners is kept; every node whose
//      owner changes goes to the step's change list; covered and fresh nodes
//      are queued per warp in lane order and published as the solid's
//      segment of the step's event list.
// k_remask follows all three, in one cooperative launch:
//   A  the change list into the owner map and the node flags (a node on the
//      rings of several solids is listed by each with the same owner; flag
//      bits are set and cleared atomically)
//   E  after a grid-wide barrier whose wait is bounded: every warp of the grid
//      takes events from the list: a fresh node is refilled by extrapolation
//      (Sec. IV.B) from nodes fluid at t and at t+1; each event's momentum and
//      torque go to its own slot; the moving solids' state becomes t+1; the
//      clock advances.
//
// Work per solid follows its perimeter: the nodes near the ends of the disk's
// chord in every row (FP32 bounds with a one-node margin) are dealt out to
// the warp's lanes, each lane fetching several nodes before it processes
// them; every decision is taken by the exact test.
//
// Precision: per-link products and each lane's running sum over its links
// (a handful) are in the arithmetic precision of the storage mode (FP32 in the
// deviation modes); the sums across lanes, the booked momenta and the motion
// are FP64, in a fixed order.  (GB300 runs FP64 at about two fused
// multiply-adds per clock per SM: FP64 lane sums would cost the force kernel
// about 100 us per step on 2000 disks.)
#include "lbm_internal.cuh"

namespace gbm {

namespace {

constexpr int SW_BLOCK = 256;
constexpr int WARPS = SW_BLOCK / 32;
constexpr double PI = 3.14159265358979323846;
constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------- barrier

// Grid-wide barrier for a cooperative launch.  Returns false (and raises
// status bit 2) if the other blocks did not arrive within p.spin_limit polls;
// the caller's block then returns, and so does every block at its next
// barrier.  A limit of 0 gives up at once: the barrier never completes (the
// time-out path's test).  The arrival count is left as it stands; the host
// clears it when it reads bit 2.
__device__ bool grid_sync(const StepParams &p) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = p.bar + 1;
        const unsigned int g = *gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(p.bar, 1u) + 1u;
        ok = 1;
        if (arrived == gridDim.x && p.spin_limit > 0) {
            atomicExch(p.bar, 0u);
            __threadfence();
            atomicAdd(p.bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*gen == g) {
                if (++spins > p.spin_limit) {
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

template <class T, int N>
__device__ __forceinline__ void warp_sum(T (&v)[N]) {
#pragma unroll
    for (int k = 0; k < N; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(FULL, v[k], o);
}

// Set or clear one bit of a 16-bit flags word atomically.
__device__ __forceinline__ void flag_bit(uint16_t *flags, long long k, int bit, bool on) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(flags + k);
    unsigned int *w = reinterpret_cast<unsigned int *>(a & ~uintptr_t(3));
    const unsigned int m = (1u << bit) << ((a & 2) ? 16 : 0);
    if (on) atomicOr(w, m);
    else atomicAnd(w, ~m);
}

__device__ __forceinline__ double cvt_s(double v) { return v; }
__device__ __forceinline__ float cvt_s(float v) { return v; }
__device__ __forceinline__ float cvt_s(__half v) { return __half2float(v); }

// Centre split into an integer part and an FP32 fraction, for FP32 bounds
// on the nodes of a row that lie within some radius of it.
struct Centre {
    int xi, yi;
    float fx, fy;
    __device__ __forceinline__ Centre(int xi_, int yi_, float fx_, float fy_)
        : xi(xi_), yi(yi_), fx(fx_), fy(fy_) {}
    __device__ __forceinline__ Centre(double X, double Y) {
        const double a = floor(X), b = floor(Y);
        xi = (int)a;
        yi = (int)b;
        fx = (float)(X - a);
        fy = (float)(Y - b);
    }
    // The integers of row j within rr of the centre, [a, b] (a > b: none),
    // from the FP32 chord; false when the row misses the circle.
    __device__ __forceinline__ bool chord(int j, float rr, int &a, int &b) const {
        const float dy = (float)(j - yi) - fy;
        const float h2 = rr * rr - dy * dy;
        if (h2 < 0.f) return false;
        const float h = sqrtf(h2);
        a = xi + (int)ceilf(fx - h);
        b = xi + (int)floorf(fx + h);
        return true;
    }
    // Unwrapped x-range [a, b] containing every node of row j within rr of
    // the centre (one node of margin on each side); false if none can be.
    __device__ __forceinline__ bool span(int j, float rr, int &a, int &b) const {
        const float dy = (float)(j - yi) - fy;
        const float h2 = rr * rr - dy * dy;
        if (h2 < 0.f) return false;
        const float h = sqrtf(h2);
        a = xi + (int)floorf(fx - h) - 1;
        b = xi + (int)ceilf(fx + h) + 1;
        return true;
    }
};

// Cell of the neighbour (x + dx, y + dy) of an in-domain node (|dx|, |dy|
// <= 3), or -1 beyond a non-periodic edge.
__device__ __forceinline__ int neighbour(const Lattice &L, int x, int y, int dx, int dy) {
    x += dx;
    y += dy;
    if (x < 0 || x >= L.nx) {
        if (L.bc_x != LBM_PERIODIC) return -1;
        x += x < 0 ? L.nx : -L.nx;
    }
    if (y < 0 || y >= L.ny) {
        if (L.bc_y != LBM_PERIODIC) return -1;
        y += y < 0 ? L.ny : -L.ny;
    }
    return y * L.pitch + x;
}

// Unwrapped node coordinates near one disk -> domain nodes, without integer
// division: along a periodic axis the nodes within WRAP_REACH of the centre
// lie within one period of the image offset taken once per disk (the domain
// is wider than 2 r + 8).
constexpr int WRAP_REACH = 8;
__host__ __device__ __forceinline__ int floor_div(int a, int n) {
    return a >= 0 ? a / n : -((n - 1 - a) / n);
}
struct Wrap {
    int ox, oy, nx, ny;
    bool px, py;
    // ix, iy = floor of the centre, rc = ceil(r)
    __device__ __forceinline__ Wrap(const Lattice &L, int ix, int iy, int rc) {
        nx = L.nx;
        ny = L.ny;
        px = L.bc_x == LBM_PERIODIC;
        py = L.bc_y == LBM_PERIODIC;
        ox = px ? nx * floor_div(ix - rc - WRAP_REACH, nx) : 0;
        oy = py ? ny * floor_div(iy - rc - WRAP_REACH, ny) : 0;
    }
    __device__ __forceinline__ bool operator()(int i, int j, int &x, int &y) const {
        x = i - ox;
        y = j - oy;
        if (px) {
            while (x >= nx) x -= nx;  // at most twice
        } else if ((unsigned)x >= (unsigned)nx) {
            return false;
        }
        if (py) {
            while (y >= ny) y -= ny;
        } else if ((unsigned)y >= (unsigned)ny) {
            return false;
        }
        return true;
    }
};

// Up to two x-ranges of a row; the second is empty when a1 > b1.
struct Ranges {
    int a0, b0, a1, b1;
};

// Nodes of row j that can lie inside exactly one of two disks of radius r
// centred at c0 and c1: between the chord ends of radius r + RING_EPS (a
// superset of each disk's nodes in the row) and those of r - RING_EPS (a
// subset), at the left and at the right.  RING_EPS is far above the FP32
// rounding of a chord end (a few 1e-3 where the chord is short), so the exact
// boundary node of each disk lies between the two; the exact test decides.
constexpr float RING_EPS = 0.05f;
__device__ __forceinline__ bool ring_ranges(const Centre &c0, const Centre &c1, float r, int j,
                                            Ranges &R) {
    int a0, b0, a1, b1, p0, q0, p1, q1;
    bool h0 = c0.chord(j, r + RING_EPS, a0, b0), h1 = c1.chord(j, r + RING_EPS, a1, b1);
    h0 = h0 && a0 <= b0;
    h1 = h1 && a1 <= b1;
    if (!h0 && !h1) return false;
    R.a1 = 1;
    R.b1 = 0;
    const bool i0 = h0 && c0.chord(j, r - RING_EPS, p0, q0) && p0 <= q0;
    const bool i1 = h1 && c1.chord(j, r - RING_EPS, p1, q1) && p1 <= q1;
    if (!i0 || !i1) {  // the row is near the top or bottom of a disk: the whole union
        R.a0 = h0 ? (h1 ? min(a0, a1) : a0) : a1;
        R.b0 = h0 ? (h1 ? max(b0, b1) : b0) : b1;
        return true;
    }
    R.a0 = min(a0, a1);
    R.b0 = max(p0, p1) - 1;  // left: first node of the outer chords .. last before the inner
    R.a1 = min(q0, q1) + 1;  // right: after the inner chords .. last of the outer
    R.b1 = max(b0, b1);
    if (R.a1 <= R.b0 + 1) {  // the two ends meet: one range
        R.b0 = R.b1;
        R.a1 = 1;
        R.b1 = 0;
    }
    return true;
}

// Nodes of row j that can be fluid nodes linked to a disk of radius r:
// r < distance <= r + sqrt(2), bounded by the chords of radius r and r + 1.5.
__device__ __forceinline__ bool annulus_ranges(const Centre &c, float r, int j, Ranges &R) {
    int ao, bo, ai, bi;
    if (!c.span(j, r + 1.5f, ao, bo)) return false;
    if (!c.span(j, r - 0.01f, ai, bi)) {
        R.a0 = ao;
        R.b0 = bo;
        R.a1 = 1;
        R.b1 = 0;
        return true;
    }
    R.a0 = ao;
    R.b0 = ai + 2;
    R.a1 = bi - 2;
    R.b1 = bo;
    if (R.a1 <= R.b0 + 1) {
        R.b0 = R.b1;
        R.a1 = 1;
        R.b1 = 0;
    }
    return true;
}

// Rows a disk can touch at either of two centres (floor iy0, iy1; rc =
// ceil(r)), with a margin of g: a superset of rows_of's.
__device__ __forceinline__ void rows_of_i(int iy0, int iy1, int rc, int g, int &j0, int &j1) {
    j0 = min(iy0, iy1) - rc - g;
    j1 = max(iy0, iy1) + rc + 1 + g;
}

// Deals the nodes of rows j0..j1 (the ranges that rng(j, R) gives for each
// row) to the lanes of the warp, U nodes per lane at a time: fetch(i, j, u)
// is called for all U nodes of a lane first (to issue their loads together),
// then mid(ok) once (loads that depend on what fetch loaded, for all U nodes
// together), then process(u, ok) for each, on every lane of the warp together
// (ok is false for items past the end and for nodes fetch rejected).  Rows come in
// blocks of RB <= 32 (lane l < RB takes row l of a block); with nw > 1 warps
// sharing the rows, this warp (wi) takes the blocks wi, wi + nw ...
struct NoMid {
    template <int NB>
    __device__ __forceinline__ void operator()(const bool (&)[NB]) const {}
};

template <int NB, int RB = 32, class RF, class FF, class PF, class MF = NoMid>
__device__ __forceinline__ void warp_nodes_n(int j0, int j1, int lane, RF &&rng, FF &&fetch,
                                             PF &&process, int wi = 0, int nw = 1,
                                             MF &&mid = MF()) {
    for (int jb = j0 + RB * wi; jb <= j1; jb += RB * nw) {
        const int j = jb + lane;
        Ranges R;
        R.a0 = R.a1 = 0;
        int n0 = 0, n1 = 0;
        if (lane < RB && j <= j1 && rng(j, R)) {
            n0 = R.b0 >= R.a0 ? R.b0 - R.a0 + 1 : 0;
            n1 = R.b1 >= R.a1 ? R.b1 - R.a1 + 1 : 0;
        }
        int inc = n0 + n1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += v;
        }
        const int total = __shfl_sync(FULL, inc, 31);
        const int excl = inc - (n0 + n1);
        for (int e0 = 0; e0 < total; e0 += 32 * NB) {
            bool ok[NB];
#pragma unroll
            for (int u = 0; u < NB; u++) {
                const int e = e0 + u * 32 + lane;
                // lane q holding item e: the last lane whose prefix is <= e
                int q = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int c = q + step;
                    const int ex = __shfl_sync(FULL, excl, c & 31);
                    if (c < 32 && ex <= e) q = c;
                }
                const int qa0 = __shfl_sync(FULL, R.a0, q), qa1 = __shfl_sync(FULL, R.a1, q);
                const int qn0 = __shfl_sync(FULL, n0, q), qex = __shfl_sync(FULL, excl, q);
                const int tt = e - qex;
                const int i = tt < qn0 ? qa0 + tt : qa1 + (tt - qn0);
                ok[u] = e < total && fetch(i, jb + q, u);
            }
            mid(ok);
#pragma unroll
            for (int u = 0; u < NB; u++) process(u, ok[u]);
        }
    }
}


// ------------------------------------------------------------- forces

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

// R(t+1) split, reduced into the domain (through the integer part: no FP64
// division) and in FP32.
__device__ __forceinline__ void set_next_centre(const Lattice &L, DSolid &b) {
    split_coord(b.xn, b.ix1, b.fx1);
    split_coord(b.yn, b.iy1, b.fy1);
    b.xnw = L.bc_x == LBM_PERIODIC ? b.xn - (double)(L.nx * floor_div(b.ix1, L.nx)) : b.xn;
    b.ynw = L.bc_y == LBM_PERIODIC ? b.yn - (double)(L.ny * floor_div(b.iy1, L.ny)) : b.yn;
    b.xnf = (float)b.xn;
    b.ynf = (float)b.yn;
}

// Motion t -> t+1 of solid s; fg = force and torque at t (lane 0): Eq. 5,
// or Eq. 4 when the context asks for the conventional form.
// The lubrication sum runs over the lanes of the warp.
__device__ void move_solid(const StepParams &p, int s, int lane, long long t, const double *fg) {
    DSolid &b = p.S[s];
    const Lattice &L = p.L;
    if (b.motion == LBM_PRESCRIBED) {
        if (lane == 0) {
            const double dt = (double)(t + 1 - b.ta);
            b.xn = __dadd_rn(b.xa, __dmul_rn(b.vx, dt));
            b.yn = __dadd_rn(b.ya, __dmul_rn(b.vy, dt));
            set_next_centre(L, b);
            b.vxn = b.vx;
            b.vyn = b.vy;
            b.omn = b.om;
        }
        return;
    }
    double fl[2] = {0.0, 0.0};
    if (p.lub > 0.0) {
        const double ka = net_weight(p, b);
        for (int q = lane; q < p.nsolid; q += 32) {
            if (q == s) continue;
            const DSolid &B = p.S[q];
            const double dx = min_image(b.x - B.x, L.nx, L.bc_x == LBM_PERIODIC);
            const double dy = min_image(b.y - B.y, L.ny, L.bc_y == LBM_PERIODIC);
            const double d = sqrt(dx * dx + dy * dy);
            const double kb = net_weight(p, B);
            const double m = lub_mag(ka > kb ? ka : kb, p.lub, d - b.r - B.r);
            if (m > 0.0 && d > 0.0) {
                fl[0] += m * dx / d;
                fl[1] += m * dy / d;
            }
        }
        warp_sum(fl);
        if (lane == 0) {
            if (L.bc_y == LBM_WALL) {
                fl[1] += lub_mag(ka, p.lub, (b.y - b.r) + 0.5);
                fl[1] -= lub_mag(ka, p.lub, ((double)L.ny - 0.5) - (b.y + b.r));
            }
            if (L.bc_x == LBM_WALL) {
                fl[0] += lub_mag(ka, p.lub, (b.x - b.r) + 0.5);
                fl[0] -= lub_mag(ka, p.lub, ((double)L.nx - 0.5) - (b.x + b.r));
            }
        }
    }
    if (lane != 0) return;
    const double M = b.rho_s * PI * b.r * b.r;
    const double I = 0.5 * M * b.r * b.r;
    const double buoy = 1.0 - p.rho0 / b.rho_s;
    const double Fx = fg[0] + buoy * M * p.grav_x + fl[0];
    const double Fy = fg[1] + buoy * M * p.grav_y + fl[1];
    const double vx1 = b.vx + Fx / M, vy1 = b.vy + Fy / M;
    b.xn = b.x + 0.5 * (b.vx + vx1);
    b.yn = b.y + 0.5 * (b.vy + vy1);
    set_next_centre(L, b);
    b.vxn = vx1;
    b.vyn = vy1;
    b.omn = b.om + fg[2] / I;
}

// Link sums of solid s at time t (populations f of time t), acc = Eq. 4
// force and torque, then Eq. 5, summed over the warp (warp wi of nw sharing
// the disk's rows).  Per link (x_f fluid, x_f + e_i owned by s): f_i =
// f~_i(x_f), the bounced f_bb = f_i - 6 w_i rho_w (e_i . v) with v the
// solid's velocity at x_s = x_f + e_i / 2; Eq. 4 = e_i f_i - e_opp f_bb,
// Eq. 5 = (e_i - v) f_i - (e_opp - v) f_bb, torque (x_s - R) x F (Eq. 7).
// (The batch's disks take the half-way boundary.)  A candidate node's flags
// and its 9 populations are loaded together, with its 8
// neighbours' owners unless lists_ok and the solid has no other solid within
// reach (then every solid neighbour of the annulus is the solid's own: a
// solid q holding a node within r_s + 4 of s's centre is in s's near list).
template <int P, bool LOCAL>
__device__ void forces_sum(const StepParams &p, int s, int lane, const void *f, int wi, int nw,
                           bool lists_ok, double (&acc)[6]) {
    using C = typename Prec<P>::C;
    using S = typename Prec<P>::S;
    constexpr int UF = 2;  // candidates a lane takes at once
    // with rho_w = rho0 and the half-way boundary a link needs only f_i of its
    // own direction: the flags come first and only the bounced directions'
    // populations (and owners) are read; otherwise all nine with the flags
    constexpr bool SPARSE = !LOCAL;
    const DSolid &b = p.S[s];
    const Lattice &L = p.L;
    const S *fs = static_cast<const S *>(f);
    const double X = b.x, Y = b.y;
    const Centre c(b.ix0, b.iy0, b.fx0, b.fy0);
    const C vx = pick<C>(b.vx, b.vxf), vy = pick<C>(b.vy, b.vyf), om = pick<C>(b.om, b.omf);
    const C rho0 = pick<C>(p.rho0, p.rho0_f);
    const int plane = (int)L.plane;
    const float r = sqrtf(b.r2f);
    const bool owners = !lists_ok || b.near_n != 0;
    const bool px = L.bc_x == LBM_PERIODIC, py = L.bc_y == LBM_PERIODIC;
    const Wrap wrap(L, b.ix0, b.iy0, b.rc);
    int j0, j1;
    rows_of_i(b.iy0, b.iy0, b.rc, 3, j0, j1);
    C lacc[6] = {0, 0, 0, 0, 0, 0};  // this lane's links
    int ii[UF], jj[UF], kk[UF];
    uint16_t fl[UF];
    uint16_t own[UF][9];
    S fv[UF][9];
    // is x_f + e_i (in the domain) a node of solid s?  own holds the owners
    // when they were read; else the flag bit suffices (no other solid in reach)
    auto linked = [&](int u, int i) -> bool {
        if (!((fl[u] >> opp(i)) & 1u)) return false;  // x_f + e_i is not solid
        if (owners) return own[u][i] == (uint16_t)s;
        return (px || (unsigned)(ii[u] + cx(i)) < (unsigned)L.nx) &&
               (py || (unsigned)(jj[u] + cy(i)) < (unsigned)L.ny);  // not beyond a wall
    };
    warp_nodes_n<UF, 16>(
        j0, j1, lane, [&](int j, Ranges &R) { return annulus_ranges(c, r, j, R); },
        [&](int iu, int j, int u) {
            int x, y;
            if (!wrap(iu, j, x, y)) return false;
            const int k = (int)cell_of(L, x, y);
            ii[u] = iu;
            jj[u] = j;
            kk[u] = k;
            fl[u] = p.flags[k];
            if (!SPARSE) {
#pragma unroll
                for (int q = 0; q < 9; q++) fv[u][q] = fs[q * plane + k];
                if (owners) {
#pragma unroll
                    for (int i = 1; i < 9; i++) {
                        const int kb = neighbour(L, x, y, cx(i), cy(i));
                        own[u][i] = kb >= 0 ? p.owner[kb] : FLUID;
                    }
                }
            }
            return true;
        },
        [&](int u, bool ok) {
            const uint16_t m = fl[u];
            if (!ok || (m & 1u) || !(m & 0x1FEu)) return;
            const int iu = ii[u], j = jj[u];
            C rho_w = rho0;
            if (LOCAL) {
                C a = 0;
#pragma unroll
                for (int q = 0; q < 9; q++) a += (C)cvt_s(fv[u][q]);
                rho_w = Prec<P>::dev ? (C)1 + a : a;
            }
#pragma unroll
            for (int i = 1; i < 9; i++) {
                if (!linked(u, i)) continue;
                C dx, dy;
                C fi = (C)cvt_s(fv[u][i]);
                if (Prec<P>::dev) fi += wgt<C>(i);
                // x_s = x_f + e_i / 2 relative to R, from the unwrapped coordinate
                if (Prec<P>::dev) {
                    dx = (C)(iu - c.xi) + (C)(0.5f * cx(i)) - (C)c.fx;
                    dy = (C)(j - c.yi) + (C)(0.5f * cy(i)) - (C)c.fy;
                } else {
                    dx = (C)(((double)iu + 0.5 * cx(i)) - X);
                    dy = (C)(((double)j + 0.5 * cy(i)) - Y);
                }
                const C ux = vx - om * dy, uy = vy + om * dx;
                const C fbb = fi - (C)6 * wgt<C>(i) * rho_w * ((C)cx(i) * ux + (C)cy(i) * uy);
                const C cmx = (C)cx(i) * fi - (C)cx(opp(i)) * fbb;
                const C cmy = (C)cy(i) * fi - (C)cy(opp(i)) * fbb;
                const C gmx = ((C)cx(i) - ux) * fi - ((C)cx(opp(i)) - ux) * fbb;
                const C gmy = ((C)cy(i) - uy) * fi - ((C)cy(opp(i)) - uy) * fbb;
                lacc[0] += cmx;
                lacc[1] += cmy;
                lacc[2] += dx * cmy - dy * cmx;
                lacc[3] += gmx;
                lacc[4] += gmy;
                lacc[5] += dx * gmy - dy * gmx;
            }
        },
        wi, nw,
        [&](const bool (&ok)[UF]) {
            if (!SPARSE) return;
            // the bounced directions of every fluid candidate, for all of them together
#pragma unroll
            for (int u = 0; u < UF; u++) {
                const uint16_t m = fl[u];
                if (!ok[u] || (m & 1u) || !(m & 0x1FEu)) continue;
                int x = 0, y = 0;
                if (owners) wrap(ii[u], jj[u], x, y);
#pragma unroll
                for (int i = 1; i < 9; i++) {
                    if (!((m >> opp(i)) & 1u)) continue;
                    fv[u][i] = fs[i * plane + kk[u]];
                    if (owners) {
                        const int kb = neighbour(L, x, y, cx(i), cy(i));
                        own[u][i] = kb >= 0 ? p.owner[kb] : FLUID;
                    }
                }
            }
        });
#pragma unroll
    for (int q = 0; q < 6; q++) acc[q] = (double)lacc[q];
    warp_sum(acc);
}

// Force record of time t of solid s from its link sums acc and the momentum
// booked into t by the node-type changes of the previous step (lane 0: Eq. 4
// force and torque, then Eq. 5); then its motion to t+1.
__device__ void record_forces(const StepParams &p, int s, int lane, long long t,
                              const double (&acc)[6], const double (&booked)[6]) {
    double fg[3] = {0.0, 0.0, 0.0};
    if (lane == 0) {
        const long long slot = t % p.ring_len;
        double *rc = p.ring + (slot * 2 + 0) * p.nsolid * 3 + (long long)s * 3;
        double *rg = p.ring + (slot * 2 + 1) * p.nsolid * 3 + (long long)s * 3;
        for (int q = 0; q < 3; q++) {
            rc[q] = acc[q] + booked[q];
            rg[q] = acc[3 + q] + booked[3 + q];
            fg[q] = p.motion_cme ? rc[q] : rg[q];  // the form that drives a free solid
        }
    }
    move_solid(p, s, lane, t, fg);
}

// ------------------------------------------------- force kernel (block)

// One block per solid: thread t takes the annulus candidates t, t + FB, ...
// (a candidate node x_f can have a link into the disk when r - eps < |x_f - R|
// <= r + sqrt 2 + eps: between the outer chord of each row and the inner one).
// A candidate's flags are read first, then only the populations of its
// bounced directions (all nine when rho_w is local or the boundary is
// interpolated) and, unless the solid's near list is empty, the owners of
// those directions.  Sums: per thread and over each warp's tree in the
// arithmetic precision of the storage mode, then across the block's warps in
// FP64, in warp order.  Warp 0 then records the force and moves the solid.
constexpr int FB = 128;                  // threads per solid
constexpr int FW = FB / 32;
constexpr float ANN_EPS = 0.05f;         // above the FP32 rounding of a chord end

template <int P, bool LOCAL, bool BND>
__global__ void __launch_bounds__(FB, 8) k_forces(const StepParams p) {
    using C = typename Prec<P>::C;
    using S = typename Prec<P>::S;
    constexpr bool SPARSE = !LOCAL && !BND;
    __shared__ int s_cnt[FB];          // the chunk's rows: exclusive prefix of their candidates
    __shared__ int s_lo[FB], s_i0[FB], s_i1[FB];  // row: [lo, hi] minus the inner chord [i0, i1]
    __shared__ double s_part[FW][6];
    __shared__ float s_disp;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const Lattice &L = p.L;
    const long long t = *p.t;
    const S *fs = static_cast<const S *>((t & 1) ? p.f1 : p.f0);  // populations of time t
    const int plane = (int)L.plane;
    const bool px = L.bc_x == LBM_PERIODIC, py = L.bc_y == LBM_PERIODIC;
    // the near lists hold at t unless a solid was added or changed since the
    // last pair test
    const bool lists_ok = p.near_id && ((volatile unsigned int *)p.bar)[3] == 0u;
    // the previous step's events are reached through the solids' segments;
    // the list fills again in this step's re-rasterisation
    if (blockIdx.x == 0 && tid == 0 && p.ev_len) {
        *p.ev_len = 0;
        *p.chg_len = 0;
    }
    if (tid == 0) s_disp = 0.f;
    for (int s = blockIdx.x; s < p.nsolid; s += gridDim.x) {
        DSolid &b = p.S[s];
        if (!solid_ok(b)) {
            if (tid == 0) atomicOr(p.status, 2);
            continue;
        }
        const Centre c(b.ix0, b.iy0, b.fx0, b.fy0);
        const Wrap wrap(L, b.ix0, b.iy0, b.rc);
        const float r = sqrtf(b.r2f);
        const bool owners = !lists_ok || b.near_n != 0;
        const C vx = pick<C>(b.vx, b.vxf), vy = pick<C>(b.vy, b.vyf), om = pick<C>(b.om, b.omf);
        const C rho0 = pick<C>(p.rho0, p.rho0_f);
        int j0, j1;
        rows_of_i(b.iy0, b.iy0, b.rc, 3, j0, j1);
        C lacc[6] = {0, 0, 0, 0, 0, 0};
        for (int jc = j0; jc <= j1; jc += FB) {  // rows in chunks of FB
            // candidates of row jc + tid
            int lo = 1, hi = 0, i0 = 1, i1 = 0, n = 0;
            const int j = jc + tid;
            if (j <= j1 && c.chord(j, r + 1.4143f + ANN_EPS, lo, hi) && lo <= hi) {
                n = hi - lo + 1;
                if (c.chord(j, r - ANN_EPS, i0, i1) && i0 <= i1) n -= i1 - i0 + 1;
            }
            // exclusive prefix over the block
            int inc = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(FULL, inc, o);
                if (lane >= o) inc += v;
            }
            if (lane == 31) s_cnt[wib] = inc;
            __syncthreads();
            if (tid < 32) {
                int w = tid < FW ? s_cnt[tid] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(FULL, w, o);
                    if (lane >= o) w += v;
                }
                if (tid < FW) s_cnt[tid] = w;  // inclusive over warps
            }
            __syncthreads();
            const int excl = (wib ? s_cnt[wib - 1] : 0) + inc - n;
            const int total = s_cnt[FW - 1];
            __syncthreads();
            s_cnt[tid] = excl;
            s_lo[tid] = lo;
            s_i0[tid] = i0 <= i1 ? i0 : 1;  // an empty inner chord: i0 > i1
            s_i1[tid] = i0 <= i1 ? i1 : 0;
            __syncthreads();
            // candidate e -> row (binary search over the prefix) and column; every
            // thread runs the same iterations (the list append is warp-wide)
            for (int base = 0; base < total; base += FB) {
                const int e = base + tid;
                int q = 0;
#pragma unroll
                for (int step = FB / 2; step > 0; step >>= 1)
                    if (q + step < FB && s_cnt[q + step] <= e) q += step;
                const int jj = jc + q;
                int iu = s_lo[q] + (e - s_cnt[q]);
                const int a = s_i0[q], bb = s_i1[q];
                if (a <= bb && iu >= a) iu += bb - a + 1;  // step over the inner chord
                int x = 0, y = 0;
                const bool here = e < total && wrap(iu, jj, x, y);
                const int k = here ? (int)cell_of(L, x, y) : 0;
                const uint16_t m = here ? p.flags[k] : (uint16_t)1u;
                const bool bounced_node = !(m & 1u) && (m & 0x1FEu);
                if (p.list_by_forces) {
                    // the node goes to the deferred per-node path's list of step t
                    const unsigned want = __ballot_sync(FULL, bounced_node);
                    if (want) {
                        int at = 0;
                        if (lane == 0) at = atomicAdd(p.bnd + (t & 1), __popc(want));
                        at = __shfl_sync(FULL, at, 0) + __popc(want & ((1u << lane) - 1u));
                        if (bounced_node) {
                            if (at < p.bnd_cap) p.bnd[2 + at] = k;
                            else atomicOr(p.status, 16);
                        }
                    }
                }
                if (!bounced_node) continue;  // solid, or no bounced population
                S fv[9];
                uint16_t own[9];
#pragma unroll
                for (int i = 1; i < 9; i++) {
                    const bool bounced = (m >> opp(i)) & 1u;  // x_f + e_i is solid
                    if (!SPARSE || bounced) fv[i] = fs[i * plane + k];
                    if (owners && bounced) {
                        const int kb = neighbour(L, x, y, cx(i), cy(i));
                        own[i] = kb >= 0 ? p.owner[kb] : FLUID;
                    }
                }
                if (!SPARSE) fv[0] = fs[k];
                C rho_w = rho0;
                if (LOCAL) {
                    C a9 = 0;
#pragma unroll
                    for (int q9 = 0; q9 < 9; q9++) a9 += (C)cvt_s(fv[q9]);
                    rho_w = Prec<P>::dev ? (C)1 + a9 : a9;
                }
#pragma unroll
                for (int i = 1; i < 9; i++) {
                    if (!((m >> opp(i)) & 1u)) continue;  // x_f + e_i is not solid
                    if (owners) {
                        if (own[i] != (uint16_t)s) continue;
                    } else if ((!px && (unsigned)(iu + cx(i)) >= (unsigned)L.nx) ||
                               (!py && (unsigned)(jj + cy(i)) >= (unsigned)L.ny)) {
                        continue;  // beyond a wall, not a solid
                    }
                    C dx, dy, ux, uy, fbb;
                    C fi = (C)cvt_s(fv[i]);
                    if (Prec<P>::dev) fi += wgt<C>(i);
                    if (BND) {
                        // the cut at fraction q of the link, and the population that
                        // returns to x_f along e_opp by the fused kernel's
                        // interpolation (full populations; M = 6 w rho_w (e_opp . v))
                        C qf;
                        if (Prec<P>::dev) {  // FP32 from the unwrapped offset, split
                            qf = (C)link_fraction_split(iu - c.xi, jj - c.yi, c.fx, c.fy, b.r,
                                                        cx(i), cy(i));
                            dx = ((C)(iu - c.xi) - (C)c.fx) + qf * (C)cx(i);
                            dy = ((C)(jj - c.yi) - (C)c.fy) + qf * (C)cy(i);
                            ux = (C)b.vxf - (C)b.omf * dy;
                            uy = (C)b.vyf + (C)b.omf * dx;
                        } else {
                            const double qd = link_fraction(L, b, x, y, i);
                            double vxd, vyd, ddx, ddy;
                            point_velocity(L, b.x, b.y, b.vx, b.vy, b.om, (double)x + qd * cx(i),
                                           (double)y + qd * cy(i), vxd, vyd, ddx, ddy);
                            qf = (C)qd;
                            dx = (C)ddx;
                            dy = (C)ddy;
                            ux = (C)vxd;
                            uy = (C)vyd;
                        }
                        const C mw =
                            -(C)6 * wgt<C>(i) * rho_w * ((C)cx(i) * ux + (C)cy(i) * uy);
                        C fo = (C)cvt_s(fv[opp(i)]);
                        if (Prec<P>::dev) fo += wgt<C>(i);
                        const C q2 = (C)2 * qf;
                        if (q2 >= (C)1) {
                            fbb = (fi + mw) / q2 + ((q2 - (C)1) / q2) * fo;
                        } else if (!((m >> i) & 1u)) {  // x_f - e_i is a fluid node
                            int xn, yn;
                            locate(L, x - cx(i), y - cy(i), xn, yn);
                            C fn = (C)cvt_s(fs[i * plane + (int)cell_of(L, xn, yn)]);
                            if (Prec<P>::dev) fn += wgt<C>(i);
                            fbb = q2 * fi + ((C)1 - q2) * fn + mw;
                        } else {
                            fbb = fi + mw;
                        }
                    } else {
                        // x_s = x_f + e_i / 2 relative to R, from the unwrapped coordinate
                        if (Prec<P>::dev) {
                            dx = (C)(iu - c.xi) + (C)(0.5f * cx(i)) - (C)c.fx;
                            dy = (C)(jj - c.yi) + (C)(0.5f * cy(i)) - (C)c.fy;
                        } else {
                            dx = (C)(((double)iu + 0.5 * cx(i)) - b.x);
                            dy = (C)(((double)jj + 0.5 * cy(i)) - b.y);
                        }
                        ux = vx - om * dy;
                        uy = vy + om * dx;
                        fbb = fi - (C)6 * wgt<C>(i) * rho_w * ((C)cx(i) * ux + (C)cy(i) * uy);
                    }
                    const C cmx = (C)cx(i) * fi - (C)cx(opp(i)) * fbb;
                    const C cmy = (C)cy(i) * fi - (C)cy(opp(i)) * fbb;
                    const C gmx = ((C)cx(i) - ux) * fi - ((C)cx(opp(i)) - ux) * fbb;
                    const C gmy = ((C)cy(i) - uy) * fi - ((C)cy(opp(i)) - uy) * fbb;
                    lacc[0] += cmx;
                    lacc[1] += cmy;
                    lacc[2] += dx * cmy - dy * cmx;
                    lacc[3] += gmx;
                    lacc[4] += gmy;
                    lacc[5] += dx * gmy - dy * gmx;
                }
            }
            __syncthreads();  // the chunk's tables are reused
        }
        warp_sum(lacc);
        if (lane == 0)
            for (int q = 0; q < 6; q++) s_part[wib][q] = (double)lacc[q];
        __syncthreads();
        if (wib == 0) {
            // lane q < 6 sums component q over the warps and over the booked
            // events, each in order; lane 0 gathers them
            double aq = 0.0, bq = 0.0;
            if (lane < 6) {
                for (int w = 0; w < FW; w++) aq += s_part[w][lane];
                if (b.ev_t == t)
                    for (int e = b.ev_off; e < b.ev_off + b.ev_n; e++) bq += p.ev_mom[6 * e + lane];
            }
            double acc[6], booked[6];
#pragma unroll
            for (int q = 0; q < 6; q++) {
                acc[q] = __shfl_sync(FULL, aq, q);
                booked[q] = __shfl_sync(FULL, bq, q);
            }
            record_forces(p, s, lane, t, acc, booked);
            if (lane == 0) {
                // distance from the centre at the last pair test, at t and t+1 (FP32
                // from the split centres, with a slack above its rounding)
                const float d0 = hypotf((float)(b.ix0 - b.ixt) + (b.fx0 - b.fxt),
                                        (float)(b.iy0 - b.iyt) + (b.fy0 - b.fyt));
                const float d1 = hypotf((float)(b.ix1 - b.ixt) + (b.fx1 - b.fxt),
                                        (float)(b.iy1 - b.iyt) + (b.fy1 - b.fyt));
                s_disp = fmaxf(s_disp, fmaxf(d0, d1) + 1e-3f);
            }
        }
        __syncthreads();  // s_part is reused
    }
    if (tid == 0 && s_disp > 0.f)  // non-negative: bits order as values
        atomicMax(p.bar + 2, __float_as_uint(s_disp));
}

// ----------------------------------------------------- re-rasterisation

// Pair test: the near list of the moving solid moving[base + warp index]
// (whole blocks call it; base + warp index may be >= nmoving).  The centres
// at t and t+1 of every solid are staged in shared memory one tile at a time.
// FP32 distances with a slack far above their rounding.
constexpr int NEAR_TILE = 512;
__device__ void phase_pairs_block(const StepParams &p, int base, int4 *ipos, float4 *fpos,
                                  float *rad) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int m = base + wib;
    const bool mine = m < p.nmoving;
    const int s = mine ? p.moving[m] : -1;
    const Lattice &L = p.L;
    const bool px = L.bc_x == LBM_PERIODIC, py = L.bc_y == LBM_PERIODIC;
    const float nxf = (float)L.nx, nyf = (float)L.ny;
    int4 bi = make_int4(0, 0, 0, 0);
    float4 bf = make_float4(0.f, 0.f, 0.f, 0.f);
    float rb = 0.f;
    if (mine) {
        const DSolid &b = p.S[s];
        rb = sqrtf(b.r2f);
        bi = make_int4(b.ix0, b.iy0, b.ix1, b.iy1);
        bf = make_float4(b.fx0, b.fy0, b.fx1, b.fy1);
    }
    uint16_t *out = mine ? p.near_id + (long long)s * NEAR_CAP : nullptr;
    int cnt = 0;
    for (int t0 = 0; t0 < p.nsolid; t0 += NEAR_TILE) {
        const int n = min(NEAR_TILE, p.nsolid - t0);
        __syncthreads();
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            const DSolid &B = p.S[t0 + q];
            ipos[q] = make_int4(B.ix0, B.iy0, B.ix1, B.iy1);
            fpos[q] = make_float4(B.fx0, B.fy0, B.fx1, B.fy1);
            rad[q] = sqrtf(B.r2f);
        }
        __syncthreads();
        if (!mine) continue;
        for (int q0 = 0; q0 < n; q0 += 32) {
            const int q = q0 + lane;
            bool hit = false;
            if (q < n && t0 + q != s) {
                const int4 ci = ipos[q];
                const float4 cf = fpos[q];
                const float lim = rb + rad[q] + NEAR_REACH + NEAR_MARGIN + 0.05f;
                float dx = (float)(bi.x - ci.x) + (bf.x - cf.x);
                float dy = (float)(bi.y - ci.y) + (bf.y - cf.y);
                float ex = (float)(bi.z - ci.z) + (bf.z - cf.z);
                float ey = (float)(bi.w - ci.w) + (bf.w - cf.w);
                if (px) {
                    dx -= nxf * rintf(dx / nxf);
                    ex -= nxf * rintf(ex / nxf);
                }
                if (py) {
                    dy -= nyf * rintf(dy / nyf);
                    ey -= nyf * rintf(ey / nyf);
                }
                hit = dx * dx + dy * dy < lim * lim || ex * ex + ey * ey < lim * lim;
            }
            const unsigned h = __ballot_sync(FULL, hit);
            if (hit) {
                const int at = cnt + __popc(h & ((1u << lane) - 1u));
                if (at < NEAR_CAP) out[at] = (uint16_t)(t0 + q);
            }
            cnt += __popc(h);
        }
    }
    if (mine && lane == 0) p.S[s].near_n = cnt <= NEAR_CAP ? cnt : -1;
}

// Is the domain node (x, y) inside the disk (X, Y, r)?  Decided at the
// node's periodic image nearest to the centre, by the exact test, as the
// rasterisation of the disk decides it.
__device__ __forceinline__ bool inside_at(const Lattice &L, int x, int y, double X, double Y,
                                          double r) {
    // the image shift in FP32: it only has to be right for nodes within r + 1
    // of the centre, far from the half-period where it could round either way
    int i = x, j = y;
    if (L.bc_x == LBM_PERIODIC) i += L.nx * (int)rintf((float)(X - (double)x) / (float)L.nx);
    if (L.bc_y == LBM_PERIODIC) j += L.ny * (int)rintf((float)(Y - (double)y) / (float)L.ny);
    const float dx = (float)((double)i - X), dy = (float)((double)j - Y), rr = (float)r + 1.0f;
    if (dx * dx + dy * dy > rr * rr) return false;
    return inside_disk(i, j, X, Y, r);
}

// Lowest-id owners of the domain node (x, y) at t (was) and t+1 (now), given
// those of solid s alone: the solids of s's near list (every solid when the
// list overflowed) that hold the node.  Centres at t: x, y (phase R only).
__device__ void near_owners(const StepParams &p, const DSolid &b, int s, int x, int y,
                            uint16_t &was, uint16_t &now) {
    const int nn = b.near_n;
    if (nn == 0) return;
    const uint16_t *nl = p.near_id + (long long)s * NEAR_CAP;
    const int n = nn < 0 ? p.nsolid : nn;
    for (int k = 0; k < n; k++) {
        const int q = nn < 0 ? k : (int)nl[k];
        if (q == s || (q >= (int)was && q >= (int)now)) continue;
        const DSolid &B = p.S[q];
        if (q < (int)was && inside_at(p.L, x, y, B.x, B.y, B.r)) was = (uint16_t)q;
        if (q < (int)now && inside_at(p.L, x, y, B.xn, B.yn, B.r)) now = (uint16_t)q;
    }
}

// Was the domain node (x, y) inside a solid of s's near list at t?  Only
// those (and s itself, tested by the caller) can have held a node within
// NEAR_REACH of s's surface.  Centres at t: xo, yo (phase E).
__device__ bool near_at_t(const StepParams &p, const DSolid &b, int s, int x, int y) {
    const int nn = b.near_n;
    if (nn == 0) return false;
    const uint16_t *nl = p.near_id + (long long)s * NEAR_CAP;
    const int n = nn < 0 ? p.nsolid : nn;
    for (int k = 0; k < n; k++) {
        const int q = nn < 0 ? k : (int)nl[k];
        if (q == s) continue;
        const DSolid &B = p.S[q];
        if (inside_at(p.L, x, y, B.xo, B.yo, B.r)) return true;
    }
    return false;
}

constexpr int EVENTS = SOLID_EVENTS;

// Ring of solid s (phase R): every node whose owner changes, into the
// step's change list, and the covered and fresh nodes of s, queued per warp
// in lane order and published as the solid's segment of the step's event
// list (to be booked into the force record of t+1), each with its unwrapped
// coordinates in the solid's frame.  No memory is read per node: the owners
// come from the geometry.
__device__ void phase_ring(const StepParams &p, int s, int lane, long long t, int2 *queue,
                           int &qn) {
    DSolid &b = p.S[s];
    const Lattice &L = p.L;
    const DiskTest in0(b.x, b.y, b.r, b.ix0, b.iy0, b.fx0, b.fy0, b.r2f, b.rmf);
    const DiskTest in1(b.xn, b.yn, b.r, b.ix1, b.iy1, b.fx1, b.fy1, b.r2f, b.rmf);
    const Centre c0(b.ix0, b.iy0, b.fx0, b.fy0), c1(b.ix1, b.iy1, b.fx1, b.fy1);
    const Wrap wrap(L, b.ix0, b.iy0, b.rc);
    const float rf = sqrtf(b.r2f);
    int j0, j1;
    rows_of_i(b.iy0, b.iy1, b.rc, 1, j0, j1);
    if (lane == 0) qn = 0;
    __syncwarp();
    constexpr int UR = 2;  // nothing is loaded per node: a short batch suffices
    int kk[UR], iu[UR], ju[UR];
    bool w0[UR];  // on the ring the node is inside s at t (true) or at t+1 (false)
    warp_nodes_n<UR>(
        j0, j1, lane, [&](int j, Ranges &R) { return ring_ranges(c0, c1, rf, j, R); },
        [&](int i, int j, int u) {
            const bool a = in0(i, j);
            if (a == in1(i, j)) return false;
            int x, y;
            if (!wrap(i, j, x, y)) return false;
            kk[u] = (int)cell_of(L, x, y);
            iu[u] = i;
            ju[u] = j;
            w0[u] = a;
            return true;
        },
        [&](int u, bool ok) {
            bool covered = false, fresh = false, changed = false;
            int2 chg;
            const int k = kk[u];
            if (ok) {
                uint16_t was = w0[u] ? (uint16_t)s : FLUID, now = w0[u] ? FLUID : (uint16_t)s;
                const int x = k % L.pitch, y = k / L.pitch;
                near_owners(p, b, s, x, y, was, now);
                if (was != now) {
                    // the new owner; bit 16: the node's solidity flips, bit 17: to solid
                    const bool sn = now != FLUID;
                    chg = make_int2(k, (int)now | (sn != (was != FLUID) ? (sn ? 0x30000 : 0x10000)
                                                                         : 0));
                    changed = true;
                }
                covered = was == FLUID && now == (uint16_t)s;
                fresh = was == (uint16_t)s && now == FLUID;
            }
            // the change list, one atomic per warp
            const unsigned cm = __ballot_sync(FULL, changed);
            if (cm) {
                int cb = 0;
                if (lane == 0) cb = atomicAdd(p.chg_len, __popc(cm));
                cb = __shfl_sync(FULL, cb, 0);
                if (changed) {
                    const int at = cb + __popc(cm & ((1u << lane) - 1u));
                    if (at < p.chg_cap) p.chg[at] = chg;
                    else atomicOr(p.status, 8);
                }
            }
            // queue the covered and fresh nodes in lane order
            __syncwarp();
            const unsigned want = __ballot_sync(FULL, covered || fresh);
            if (!want) return;
            const int base = qn;
            __syncwarp();
            if (lane == 0) qn = base + __popc(want);
            if (covered || fresh) {
                const int pos = base + __popc(want & ((1u << lane) - 1u));
                // node code, and its unwrapped coordinates relative to floor(R)
                if (pos < EVENTS)
                    queue[pos] = make_int2(
                        (k << 1) | (fresh ? 1 : 0),
                        (int)((unsigned)(iu[u] - c0.xi + 32768) |
                              ((unsigned)(ju[u] - c0.yi + 32768) << 16)));
                else atomicOr(p.status, 8);
            }
            __syncwarp();
        });
    __syncwarp();
    const int n = min(qn, EVENTS);
    // publish the events: one segment of the step's event list per solid
    int off = 0;
    if (lane == 0 && n) off = atomicAdd(p.ev_len, n);
    off = __shfl_sync(FULL, off, 0);
    const bool fits = off + n <= p.ev_cap;
    for (int e = lane; e < n; e += 32) {
        if (fits) {
            const int2 q = queue[e];
            const unsigned d = (unsigned)q.y;
            p.ev[off + e] = make_int4(q.x, s, c0.xi + (int)(d & 0xFFFFu) - 32768,
                                      c0.yi + (int)(d >> 16) - 32768);
        }
    }
    if (lane == 0) {
        if (!fits) atomicOr(p.status, 8);
        b.ev_off = off;
        b.ev_n = fits ? n : 0;
        b.ev_t = t + 1;
        b.xo = b.x;
        b.yo = b.y;
        b.ixo = b.ix0;
        b.iyo = b.iy0;
        b.fxo = b.fx0;
        b.fyo = b.fy0;
    }
    __syncwarp();
}

// One covered or fresh node of the step's event list, with the whole warp
// (phase E): the refill of a fresh node (Sec. IV.B), then the node's momentum
// (covered: post-collision, into the solid; fresh: refilled, out of it) and
// its torque about the solid's new centre, into the event's slot of ev_mom.
// Events are independent: a refill reads only nodes that are fluid at t and
// at t+1, which no event writes.
template <int P>
__device__ void phase_event(const StepParams &p, int e, int lane, void *fnew) {
    using C = typename Prec<P>::C;
    using S = typename Prec<P>::S;
    const Lattice &L = p.L;
    const S *fsn = static_cast<const S *>(fnew);
    const int pl = (int)L.plane;
    const int4 ev = p.ev[e];
    const int code = ev.x, s = ev.y;
    const DSolid &b = p.S[s];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    {
        const int k = code >> 1;
        const int x = k % L.pitch, y = k / L.pitch;
        C fj = 0;  // lane j < 9: population j of the node (a fresh node's as stored)
        if (code & 1) {
            // fresh: refill (Sec. IV.B).  Lane 3(i-1)+(d-1) tests x + d e_i: a
            // node fluid at t+1 (owner map) that no solid held at t (the
            // solid's own disk at t in its frame, and its near list)
            bool use = false;
            if (lane < 24) {
                const int i = lane / 3 + 1, d = lane % 3 + 1;
                const int kp = neighbour(L, x, y, d * cx(i), d * cy(i));
                if (kp >= 0 && p.owner[kp] == FLUID) {
                    const DiskTest old(b.xo, b.yo, b.r, b.ixo, b.iyo, b.fxo, b.fyo, b.r2f,
                                       b.rmf);
                    use = !old(ev.z + d * cx(i), ev.w + d * cy(i)) &&
                          !near_at_t(p, b, s, kp % L.pitch, kp / L.pitch);
                }
            }
            const unsigned um = __ballot_sync(FULL, use);
            unsigned d3 = 0, d2 = 0, d1 = 0;  // directions old-fluid up to distance 3, 2, 1
#pragma unroll
            for (int i = 1; i < 9; i++) {
                const unsigned bits = (um >> (3 * (i - 1))) & 7u;
                if (bits == 7u) d3 |= 1u << (i - 1);
                if ((bits & 3u) == 3u) d2 |= 1u << (i - 1);
                if (bits & 1u) d1 |= 1u << (i - 1);
            }
            unsigned dirs = 0;
            int scheme = 0;  // 1: A1, 2: A2, 3: A3, 0: equilibrium
            if (p.refill <= LBM_REFILL_A1 && d3) {
                dirs = d3;
                scheme = 1;
            } else if (p.refill <= LBM_REFILL_A2 && d2) {
                dirs = d2;
                scheme = 2;
            } else if (d1) {
                dirs = d1;
                scheme = 3;
            }
            if (scheme) {
                // lane 3j + (d-1) sums f_j(x + d e_i) over the chosen directions
                const int j = lane / 3, d = lane % 3 + 1;
                const C wd = scheme == 1 ? (d == 1 ? (C)3 : (d == 2 ? (C)-3 : (C)1))
                                         : (scheme == 2 ? (d == 1 ? (C)2 : (d == 2 ? (C)-1 : (C)0))
                                                        : (d == 1 ? (C)1 : (C)0));
                C sum = 0;
                if (lane < 27 && wd != (C)0) {
#pragma unroll
                    for (int i = 1; i < 9; i++) {
                        if (!((dirs >> (i - 1)) & 1u)) continue;
                        sum += (C)ldc(fsn + j * pl + neighbour(L, x, y, d * cx(i), d * cy(i)));
                    }
                }
                C v = wd * sum;
                v += __shfl_down_sync(FULL, v, 1) + __shfl_down_sync(FULL, v, 2);
                v = stored(fsn, v / (C)__popc(dirs));
                if (lane < 27 && lane % 3 == 0) st(static_cast<S *>(fnew) + j * pl + k, v);
                fj = __shfl_sync(FULL, v, 3 * (lane < 9 ? lane : 0));  // lane j <- lane 3j
            } else if (lane < 9) {
                // no old-fluid neighbour: equilibrium at rho0 and the solid's velocity
                double ux, uy, ddx, ddy;
                point_velocity(L, b.xn, b.yn, b.vxn, b.vyn, b.omn, (double)x, (double)y, ux, uy,
                               ddx, ddy);
                const double eu = cx(lane) * ux + cy(lane) * uy, uu = ux * ux + uy * uy;
                const double fe =
                    p.rho0 * wgt<double>(lane) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
                fj = stored(fsn, (C)(Prec<P>::dev ? fe - wgt<double>(lane) : fe));
                st(static_cast<S *>(fnew) + lane * pl + k, fj);
            }
            __syncwarp();
        } else if (lane < 9) {
            fj = (C)ldc(fsn + lane * pl + k);  // covered: its post-collision populations
        }
        // momentum and mass of the node (post-collision if covered, refilled if
        // fresh), summed in the arithmetic precision of the storage mode
        C jm[3] = {0, 0, 0};
        if (lane < 9) {
            C v = fj;
            if (Prec<P>::dev) v += wgt<C>(lane);
            jm[0] = (C)cx(lane) * v;
            jm[1] = (C)cy(lane) * v;
            jm[2] = v;
        }
        warp_sum(jm);
        if (lane == 0) {
            // fresh: from the solid; covered: to it.  The node's momentum, its
            // velocity relative to the boundary and its lever about the new
            // centre in the arithmetic precision C (the FP64 mode from the
            // domain node at the nearest periodic image; the deviation modes
            // from the node's unwrapped coordinates and the split centre)
            const C sgn = (code & 1) ? (C)-1 : (C)1;
            const C mx = jm[0], my = jm[1], mm = jm[2];
            C ux, uy, dx, dy;
            if (P == LBM_FP64) {
                double vx, vy, ddx, ddy;
                point_velocity(L, b.xn, b.yn, b.vxn, b.vyn, b.omn, (double)x, (double)y, vx, vy,
                               ddx, ddy);
                ux = (C)vx;
                uy = (C)vy;
                dx = (C)ddx;
                dy = (C)ddy;
            } else {
                dx = (C)(ev.z - b.ix1) - (C)b.fx1;
                dy = (C)(ev.w - b.iy1) - (C)b.fy1;
                const C vxn = (C)b.vxn, vyn = (C)b.vyn, omn = (C)b.omn;
                ux = vxn - omn * dy;
                uy = vyn + omn * dx;
            }
            // the Eq. 5 record's booking: the same, or relative to the boundary, m (u - v)
            const C rx = p.relative_changes ? mx - mm * ux : mx;
            const C ry = p.relative_changes ? my - mm * uy : my;
            acc[0] = (double)(sgn * mx);
            acc[1] = (double)(sgn * my);
            acc[2] = (double)(sgn * (dx * my - dy * mx));
            acc[3] = (double)(sgn * rx);
            acc[4] = (double)(sgn * ry);
            acc[5] = (double)(sgn * (dx * ry - dy * rx));
        }
    }
    if (lane == 0)
        for (int q = 0; q < 6; q++) p.ev_mom[6 * e + q] = acc[q];
    __syncwarp();
}

// The state of a moving solid becomes that of t+1 (xo, yo keep R(t) for the
// events of the step).
__device__ __forceinline__ void advance_solid(const Lattice &L, DSolid &b) {
    b.x = b.xn;
    b.y = b.yn;
    b.xw = b.xnw;
    b.yw = b.ynw;
    b.ix0 = b.ix1;
    b.iy0 = b.iy1;
    b.fx0 = b.fx1;
    b.fy0 = b.fy1;
    b.xwi = L.bc_x == LBM_PERIODIC ? b.ix1 - L.nx * floor_div(b.ix1, L.nx) : b.ix1;
    b.ywi = L.bc_y == LBM_PERIODIC ? b.iy1 - L.ny * floor_div(b.iy1, L.ny) : b.iy1;
    b.xwr = b.fx1;
    b.ywr = b.fy1;
    b.vx = b.vxn;
    b.vy = b.vyn;
    b.om = b.omn;
    b.vxf = (float)b.vxn;
    b.vyf = (float)b.vyn;
    b.omf = (float)b.omn;
    b.xf = b.xnf;
    b.yf = b.ynf;
}

// P and R (beside the advection-collision kernel), one warp per moving solid.
__global__ void __launch_bounds__(SW_BLOCK, 4) k_ring(const StepParams p) {
    __shared__ int2 queue[WARPS][EVENTS];
    __shared__ int qn[WARPS];
    __shared__ int4 tile_ipos[NEAR_TILE];
    __shared__ float4 tile_fpos[NEAR_TILE];
    __shared__ float tile_rad[NEAR_TILE];
    // a barrier of an earlier launch gave up: the state is not the method's
    // any more, and this launch does nothing (the host reports the time-out)
    if (*(volatile int *)p.status & 4) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long t = *p.t;
    const volatile unsigned int *ctl = p.bar;
    // nothing changes the control words between the force kernel and k_remask
    const bool pairs = ctl[3] != 0u || __uint_as_float(ctl[2]) >= 0.5f * NEAR_MARGIN;
    if (pairs) phase_pairs_block(p, blockIdx.x * WARPS, tile_ipos, tile_fpos, tile_rad);
    const int m = blockIdx.x * WARPS + wib;
    if (m >= p.nmoving) return;
    const int s = p.moving[m];
    DSolid &b = p.S[s];
    if (pairs && lane == 0) {  // the centres the near list was taken at
        b.ixt = b.ix0;
        b.iyt = b.iy0;
        b.fxt = b.fx0;
        b.fyt = b.fy0;
    }
    __syncwarp();
    if (solid_ok(b)) phase_ring(p, s, lane, t, queue[wib], qn[wib]);
    else if (lane == 0) atomicOr(p.status, 2);
}

// A and E (after the advection-collision kernel and k_ring), one cooperative
// launch.
template <int P>
__global__ void __launch_bounds__(SW_BLOCK, 4) k_remask(const StepParams p) {
    if (*(volatile int *)p.status & 4) return;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * WARPS + wib, nw = gridDim.x * WARPS;
    const int gt = blockIdx.x * SW_BLOCK + threadIdx.x, nt = gridDim.x * SW_BLOCK;
    const Lattice &L = p.L;
    const long long t = *p.t;
    void *fnew = ((t + 1) & 1) ? p.f1 : p.f0;  // populations of time t+1
    // A: owners and flags of t+1
    const int nchg = min(*(volatile int *)p.chg_len, p.chg_cap);
    for (int c = gt; c < nchg; c += nt) {
        const int2 q = p.chg[c];
        const int k = q.x;
        p.owner[k] = (uint16_t)(q.y & 0xFFFF);
        if (q.y & 0x10000) {
            // bit 0 of the node, bit d of the neighbour x + e_d
            const bool sn = (q.y & 0x20000) != 0;
            const int x = k % L.pitch, y = k / L.pitch;
            flag_bit(p.flags, k, 0, sn);
#pragma unroll
            for (int d = 1; d < 9; d++) {
                const int kn = neighbour(L, x, y, cx(d), cy(d));
                if (kn >= 0) flag_bit(p.flags, kn, d, sn);
            }
        }
    }
    if (!grid_sync(p)) return;
    if (gt == 0) {
        *p.t = t + 1;  // every block has read t
        volatile unsigned int *ctl = p.bar;
        if (ctl[3] != 0u || __uint_as_float(ctl[2]) >= 0.5f * NEAR_MARGIN) {
            ctl[2] = 0u;  // the pair test of this step has run
            ctl[3] = 0u;
        }
    }
    // E: the step's covered and fresh nodes, dealt to every warp of the grid
    const int nev = min(*(volatile int *)p.ev_len, p.ev_cap);
    for (int e = gw; e < nev; e += nw) phase_event<P>(p, e, lane, fnew);
    for (int m = gt; m < p.nmoving; m += nt) advance_solid(L, p.S[p.moving[m]]);
}

template <int P, bool LOCAL, bool BND>
cudaError_t launch_f(const StepParams &p, cudaStream_t st) {
    static int per_sm = -1, sms = 0;
    if (per_sm < 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forces<P, LOCAL, BND>,
                                                              FB, 0);
        if (e != cudaSuccess) return e;
    }
    int blocks = p.nsolid;  // one solid per block, looped beyond the resident blocks
    if (blocks > 8 * per_sm * sms) blocks = 8 * per_sm * sms;
    if (blocks < 1) blocks = 1;
    k_forces<P, LOCAL, BND><<<blocks, FB, 0, st>>>(p);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_r(const StepParams &p, cudaStream_t st) {
    static int per_sm = -1, sms = 0;
    if (per_sm < 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_remask<P>, SW_BLOCK, 0);
        if (e != cudaSuccess) return e;
    }
    // every resident block: the changes go to every thread, the events to
    // every warp
    int blocks = per_sm * sms;
    if (blocks < 1) blocks = 1;
    StepParams pp = p;
    void *args[] = {&pp};
    return cudaLaunchCooperativeKernel((const void *)k_remask<P>, dim3(blocks), dim3(SW_BLOCK),
                                       args, 0, st);
}

// ------------------------------------------------------------- batch

// Force records of a batch of independent domains whose solids rest: one
// block per (case, solid) item of the active list, phase F only.  The last
// block to finish (a ticket, no waiting) advances the step counter of every
// active case and swaps its population buffers (batch convention: f0 holds
// the current time), after every block has read them.
template <int P, bool LOCAL>
__global__ void __launch_bounds__(SW_BLOCK, 2)
    k_solids_batch(StepParams *cases, const int2 *__restrict__ items,
                   const int *__restrict__ nitems, const int *__restrict__ active,
                   const int *__restrict__ nactive, unsigned int *ticket) {
    __shared__ bool last;
    __shared__ double part[WARPS][6];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n = *nitems;
    // one block per item: the warps share the disk's rows, then warp 0 adds
    // their sums in warp order
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int2 it = items[k];
        const StepParams &p = cases[it.x];
        const long long t = *p.t;
        const void *fcur = p.f0;  // batch convention: f0 holds time t
        if (!solid_ok(p.S[it.y])) {
            if (threadIdx.x == 0) atomicOr(p.status, 2);
            continue;
        }
        double acc[6];
        forces_sum<P, LOCAL>(p, it.y, lane, fcur, wib, WARPS, false, acc);
        if (lane == 0)
            for (int q = 0; q < 6; q++) part[wib][q] = acc[q];
        __syncthreads();
        if (wib == 0) {
            double tot[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            if (lane == 0)
                for (int w = 0; w < WARPS; w++)
                    for (int q = 0; q < 6; q++) tot[q] += part[w][q];
            const double none[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // resting: no node changes type
            record_forces(p, it.y, lane, t, tot, none);
        }
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int na = *nactive;
    for (int a = threadIdx.x; a < na; a += blockDim.x) {
        StepParams &p = cases[active[a]];
        *p.t += 1;
        void *f = p.f0;  // the populations of t+1 become the current ones
        p.f0 = p.f1;
        p.f1 = f;
    }
    if (threadIdx.x == 0) *ticket = 0;
}

template <int P, bool LOCAL>
cudaError_t launch_sb(const BatchLaunch &b, cudaStream_t st) {
    static int per_sm = -1, sms = 0;
    if (per_sm < 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solids_batch<P, LOCAL>,
                                                              SW_BLOCK, 0);
        if (e != cudaSuccess) return e;
    }
    int blocks = b.max_items;
    if (blocks > per_sm * sms) blocks = per_sm * sms;
    if (blocks < 1) blocks = 1;
    k_solids_batch<P, LOCAL><<<blocks, SW_BLOCK, 0, st>>>(b.cases, b.items, b.nitems, b.active,
                                                          b.nactive, b.ticket);
    return cudaGetLastError();
}

// Convergence test and list rebuild, one block.  Case states: 0 active,
// 1 converged, 2 step cap reached, 3 unstable (a status bit raised, or a
// non-finite drag).  The drag of a case is the x component of the Eq. 5
// force summed over its solids in the latest record; it has converged when
// it moved by less than tol relative since the previous test.  Modes:
// BATCH_TEST tests and rebuilds the lists if a case retired; BATCH_REBUILD
// keeps the states, clears the drag history and rebuilds the lists;
// BATCH_GATHER only copies the step counters.  Every mode copies them.
constexpr int CV_BLOCK = 1024;
__global__ void __launch_bounds__(CV_BLOCK)
    k_batch_converge(BatchLaunch b, int ncase, double tol, long long max_steps, int window,
                     int mode, int *state, double *drag, int *calm, double *anchor,
                     long long *steps, int *toff, int *ioff, int tile_w, int tile_h) {
    __shared__ int changed;
    __shared__ int wsum[3][CV_BLOCK / 32];
    __shared__ int carry[3];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        changed = mode == BATCH_REBUILD;
        carry[0] = carry[1] = carry[2] = 0;
    }
    __syncthreads();
    for (int c = tid; c < ncase; c += CV_BLOCK) {
        const StepParams &p = b.cases[c];
        const long long t = *p.t;
        steps[c] = t;
        if (mode == BATCH_GATHER) continue;
        if (mode == BATCH_REBUILD) {
            drag[c] = __longlong_as_double(0x7ff8000000000000ll);  // no history
            anchor[c] = drag[c];
            calm[c] = 0;
            continue;
        }
        if (state[c] != 0) continue;
        int ns = 0;
        if (*p.status != 0) ns = 3;
        double D = 0.0;
        if (ns == 0 && p.nsolid > 0 && t >= 1) {
            const long long slot = (t - 1) % p.ring_len;
            const double *rg = p.ring + (slot * 2 + 1) * p.nsolid * 3;
            for (int s = 0; s < p.nsolid; s++) D += rg[s * 3];
            // converged once the drag has stayed within tol of the drag at the
            // start of `window` tests in a row (window 1: of the previous test)
            const double a = anchor[c];
            drag[c] = D;
            if (!isfinite(D)) ns = 3;
            else if (isfinite(a) && fabs(D - a) < tol * fabs(D)) {
                if (++calm[c] >= window) ns = 1;
            } else {
                anchor[c] = D;
                calm[c] = 0;
            }
        }
        if (ns == 0 && t >= max_steps) ns = 2;
        if (ns != 0) {
            state[c] = ns;
            changed = 1;
        }
    }
    __syncthreads();
    if (!changed) return;
    // exclusive scans of (active, tiles, items) over the cases, in chunks
    for (int base = 0; base < ncase; base += CV_BLOCK) {
        const int c = base + tid;
        int v[3] = {0, 0, 0};
        if (c < ncase && state[c] == 0) {
            const Lattice &L = b.cases[c].L;
            v[0] = 1;
            v[1] = (L.nx + tile_w - 1) / tile_w * ((L.ny + tile_h - 1) / tile_h);
            v[2] = b.cases[c].nsolid;
        }
        int inc[3];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            inc[q] = v[q];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(FULL, inc[q], o);
                if (lane >= o) inc[q] += u;
            }
            if (lane == 31) wsum[q][wid] = inc[q];
        }
        __syncthreads();
        if (wid == 0) {
#pragma unroll
            for (int q = 0; q < 3; q++) {
                int w = wsum[q][lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(FULL, w, o);
                    if (lane >= o) w += u;
                }
                wsum[q][lane] = w;  // inclusive over warps
            }
        }
        __syncthreads();
        int ex[3];
#pragma unroll
        for (int q = 0; q < 3; q++) ex[q] = carry[q] + (wid ? wsum[q][wid - 1] : 0) + inc[q] - v[q];
        if (v[0]) {
            b.active[ex[0]] = c;
            toff[c] = ex[1];
            ioff[c] = ex[2];
        }
        __syncthreads();
        if (tid == 0)
            for (int q = 0; q < 3; q++) carry[q] += wsum[q][CV_BLOCK / 32 - 1];
        __syncthreads();
    }
    const int na = carry[0];
    if (tid == 0) {
        *b.nactive = na;
        *b.ntiles = carry[1];
        *b.nitems = carry[2];
    }
    int4 *tiles = b.tiles;
    int2 *items = b.items;
    for (int a = 0; a < na; a++) {
        const int c = b.active[a];
        const Lattice &L = b.cases[c].L;
        const int nbx = (L.nx + tile_w - 1) / tile_w, nby = (L.ny + tile_h - 1) / tile_h;
        const int nt = nbx * nby, o = toff[c];
        for (int k = tid; k < nt; k += CV_BLOCK)
            tiles[o + k] = make_int4(c, k % nbx, (k / nbx) * tile_h, 0);
        const int ns = b.cases[c].nsolid, oi = ioff[c];
        for (int s = tid; s < ns; s += CV_BLOCK) items[oi + s] = make_int2(c, s);
    }
}

}  // namespace

cudaError_t launch_solids_batch(const BatchLaunch &b, cudaStream_t st) {
    if (b.precision == LBM_FP64)
        return b.local ? launch_sb<LBM_FP64, true>(b, st) : launch_sb<LBM_FP64, false>(b, st);
    if (b.precision == LBM_FP32_DEV)
        return b.local ? launch_sb<LBM_FP32_DEV, true>(b, st) : launch_sb<LBM_FP32_DEV, false>(b, st);
    return b.local ? launch_sb<LBM_FP16_DEV, true>(b, st) : launch_sb<LBM_FP16_DEV, false>(b, st);
}

cudaError_t launch_batch_converge(const BatchLaunch &b, const BatchState &s, int mode,
                                  cudaStream_t st) {
    k_batch_converge<<<1, CV_BLOCK, 0, st>>>(b, s.ncase, s.tol, s.max_steps, s.window, mode,
                                             s.state, s.drag, s.calm, s.anchor, s.steps, s.toff,
                                             s.ioff, tile_nodes(b.precision, b.variant),
                                             b.tile_h);
    return cudaGetLastError();
}

cudaError_t launch_forces(const StepParams &p, cudaStream_t st) {
    if (p.nsolid == 0) return cudaSuccess;
    const bool local = p.rho_w_mode == LBM_RHOW_LOCAL, bnd = p.boundary == LBM_INTERPOLATED;
#define GBM_F(P)                                                                            \
    return local ? (bnd ? launch_f<P, true, true>(p, st) : launch_f<P, true, false>(p, st)) \
                 : (bnd ? launch_f<P, false, true>(p, st) : launch_f<P, false, false>(p, st))
    switch (p.precision) {
        case LBM_FP64: GBM_F(LBM_FP64);
        case LBM_FP32_DEV: GBM_F(LBM_FP32_DEV);
        default: GBM_F(LBM_FP16_DEV);
    }
#undef GBM_F
}

cudaError_t launch_ring(const StepParams &p, cudaStream_t st) {
    if (p.nmoving == 0) return cudaSuccess;
    k_ring<<<(p.nmoving + WARPS - 1) / WARPS, SW_BLOCK, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_remask(const StepParams &p, cudaStream_t st) {
    if (p.nmoving == 0) return cudaSuccess;
    switch (p.precision) {
        case LBM_FP64: return launch_r<LBM_FP64>(p, st);
        case LBM_FP32_DEV: return launch_r<LBM_FP32_DEV>(p, st);
        default: return launch_r<LBM_FP16_DEV>(p, st);
    }
}

}  // namespace gbm
