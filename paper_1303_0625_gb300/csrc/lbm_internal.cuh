// Internal definitions shared by the CUDA translation units of the library:
// D2Q9 tables, storage precisions, the device-side parameter block and the
// geometric helpers (disk boxes, inside test, periodic images).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm.h"

namespace gbm {

constexpr uint16_t FLUID = 0xFFFFu;   // owner value of a fluid node
constexpr int SOLID_BLOCK = 256;      // threads of the per-solid kernels
constexpr int SC_BLOCK_X = 128;       // threads of the advection-collision kernel

// D2Q9 velocities in the order of Sec. III.C of the paper:
// (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
// lattice weights 4/9, 1/9, 1/36
template <class C>
__host__ __device__ constexpr C wgt(int i) {
    return i == 0 ? C(4) / C(9) : (i <= 4 ? C(1) / C(9) : C(1) / C(36));
}

// Per-solid record on the device (array of structs).
struct DSolid {
    double xa, ya;     // position when added (prescribed motion)
    double x, y;       // centre R(t)
    double xn, yn;     // centre R(t+1), written by the force kernel of the step
    double xw, yw;     // R(t) reduced into the domain along periodic axes
    double xnw, ynw;   // R(t+1) reduced likewise
    double vx, vy, om; // V(t), Omega(t)
    double vxn, vyn, omn;
    double r, rho_s;
    double xo, yo;     // R(t) kept through the re-rasterisation (R(t) itself becomes R(t+1)
                       // there); equal to x, y between steps
    long long ev_t;    // record (time) into which the segment ev_off, ev_n books its momenta
    long long ta;      // time when added
    float vxf, vyf, omf;  // FP32 copies of vx, vy, om for the FP32 kernels
    float xf, yf, xnf, ynf;  // FP32 copies of x, y, xn, yn for the pair test
    int xwi, ywi;      // integer part of (xw, yw) ...
    float xwr, ywr;    // ... and the FP32 remainder, for FP32 lever arms
    int motion;
    int near_n;        // entries of the solid's near list (-1: too many; every solid is tested)
    int ev_off, ev_n;  // the solid's segment of the covered/fresh event list
    // Centres split into floor() and the FP32 remainder, for FP32 geometry
    // without FP64 arithmetic in the per-solid kernels: R(t), R(t+1), R(t) kept
    // through the re-rasterisation (as xo, yo), and the centre at the last
    // pair test.
    int ix0, iy0, ix1, iy1, ixo, iyo, ixt, iyt;
    float fx0, fy0, fx1, fy1, fxo, fyo, fxt, fyt;
    int rc;            // ceil(r)
    float r2f, rmf;    // (float)(r * r) and the exact test's band, 1e-5 r^2 + 1e-5
};

// floor(X) and the FP32 remainder X - floor(X) (host and device).
__host__ __device__ inline void split_coord(double X, int &i, float &f) {
    const double a = floor(X);
    i = (int)a;
    f = (float)(X - a);
}

// Near list: the solids that can own a node within NEAR_REACH (lattice
// units) of a disk's surface at t or t+1 are those whose centres are closer
// than r_s + r_q + NEAR_REACH; the list is built with a further NEAR_MARGIN
// and stays valid while every solid has moved less than NEAR_MARGIN / 2 from
// its centre at the test.  NEAR_REACH covers the re-rasterisation ring
// (within one node of the surface, plus one step of motion) and the refill's
// extrapolation nodes (three links, 3 sqrt(2) < 4.5, from a fresh node).
constexpr int NEAR_CAP = 32;
constexpr float NEAR_REACH = 4.5f;
constexpr float NEAR_MARGIN = 4.0f;

// covered/fresh nodes one solid can queue per step
constexpr int SOLID_EVENTS = 256;

struct Lattice {
    int nx, ny, pitch; // pitch = elements per row of every 2-D plane
    int bc_x, bc_y;
    long long plane;   // ny * pitch
};

struct StepParams {
    Lattice L;
    void *f0, *f1;            // population buffers; buffer (t & 1) holds time t
    uint16_t *owner, *flags;
    DSolid *S;
    int nsolid;
    const int *moving;        // ids of solids that translate (or are free)
    int nmoving;
    double *ring;             // [ring_len][2][nsolid][3], slot = time % ring_len
    int ring_len;
    long long *t;             // device step counter
    int *status;              // bit 0: non-finite or non-positive density; bit 1: bad solid state
    double tau, omega, rho0;
    double wall_ux0, wall_ux1;
    double body_x, body_y;
    double umax;
    double grav_x, grav_y, lub;
    double u0x, u0y;
    int rho_w_mode, refill, precision;
    int motion_cme;           // free solids move under Eq. 4 (1) or Eq. 5 (0)
    int relative_changes;     // Eq. 5 record books covered/fresh momenta as m (u - v)
    int collision;            // LBM_BGK or LBM_MRT
    int boundary;             // disks: LBM_HALFWAY or LBM_INTERPOLATED
    int sc_variant;           // node width per thread of the advection-collision kernel
    float omega_f, body_xf, body_yf, rho0_f;  // FP32 copies for the FP32 kernels
    float wall_ux0_f, wall_ux1_f, umax_f;
    unsigned int *bar;        // per-solid control words: grid barrier {count, generation},
                              // largest displacement since the pair test (FP32 bits), pair
                              // test requested
    long long spin_limit;     // polls of a bounded device wait (0: give up at once)
    uint16_t *near_id;        // [nsolid][NEAR_CAP] near lists
    int4 *ev;                 // covered/fresh events of the step: {node code (cell << 1 |
                              // fresh), solid, unwrapped x, y in the solid's frame}
    double *ev_mom;           // [6] momentum and torque of each event: Eq. 4, Eq. 5 booking
    int *ev_len;              // events published this step (cleared after use)
    int ev_cap;
    int2 *chg;                // owner changes of the step: {cell, new owner | bit 16: the
                              // solidity flips | bit 17: to solid}
    int *chg_len;             // changes listed this step (cleared with ev_len)
    int chg_cap;
    int *bnd;                 // deferred per-node path: {length at even t, at odd t, list...}
    int bnd_cap;              // capacity of the list
    int list_by_forces;       // the force kernel fills the deferred list; the fused pass
                              // leaves the update to launch_deferred_update
};

// Half-width of a box around floor(R) that holds every fluid node with a
// link into a disk (within r + sqrt 2 of R, R within one node of floor(R));
// the box's (2 h + 1)^2 nodes bound the disk's entries in the deferred list.
__host__ __device__ inline int boundary_half(double r) { return (int)ceil(r) + 3; }

template <class C> __device__ __forceinline__ C pick(double d, float f);
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

// ---------------------------------------------------------------- storage

template <int P> struct Prec;
template <> struct Prec<LBM_FP64> {
    using S = double;
    using C = double;
    static constexpr bool dev = false;
};
template <> struct Prec<LBM_FP32_DEV> {
    using S = float;
    using C = float;
    static constexpr bool dev = true;
};
template <> struct Prec<LBM_FP16_DEV> {
    using S = __half;
    using C = float;
    static constexpr bool dev = true;
};

__device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ double ldc(const double *p) { return *p; }
__device__ __forceinline__ float ldc(const float *p) { return *p; }
__device__ __forceinline__ float ldc(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void st(double *p, double v) { *p = v; }
__device__ __forceinline__ void st(float *p, float v) { *p = v; }
__device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
__device__ __forceinline__ void st(float *p, double v) { *p = (float)v; }
// v rounded to the storage type S, as st() stores it, in the arithmetic type
__device__ __forceinline__ double stored(const double *, double v) { return v; }
__device__ __forceinline__ float stored(const float *, float v) { return v; }
__device__ __forceinline__ float stored(const __half *, float v) {
    return __half2float(__float2half_rn(v));
}
__device__ __forceinline__ void st(__half *p, double v) { *p = __double2half(v); }

// Population i of cell k as an FP64 value f_i (undoing the deviation storage).
template <int P>
__device__ __forceinline__ double f64(const void *buf, long long plane, int i, long long k) {
    using S = typename Prec<P>::S;
    double v = (double)ldc(static_cast<const S *>(buf) + (long long)i * plane + k);
    if (Prec<P>::dev) v += wgt<double>(i);
    return v;
}
// Store an FP64 population value f_i into the storage precision.
template <int P>
__device__ __forceinline__ void put64(void *buf, long long plane, int i, long long k, double v) {
    using S = typename Prec<P>::S;
    if (Prec<P>::dev) v -= wgt<double>(i);
    st(static_cast<S *>(buf) + (long long)i * plane + k, v);
}

// --------------------------------------------------------------- geometry

struct Box {
    int x0, y0, w, h;
};

// Nodes whose integer coordinates can be inside the disk, grown by g.
__device__ __forceinline__ Box disk_box(double X, double Y, double r, int g) {
    Box b;
    b.x0 = (int)floor(__dsub_rn(X, r)) - g;
    b.y0 = (int)floor(__dsub_rn(Y, r)) - g;
    b.w = (int)ceil(__dadd_rn(X, r)) + g - b.x0 + 1;
    b.h = (int)ceil(__dadd_rn(Y, r)) + g - b.y0 + 1;
    return b;
}

// A solid whose centre is not finite (or absurdly far away) would give a
// meaningless box; per-solid kernels skip it and raise status bit 1.
__device__ __forceinline__ bool solid_ok(const DSolid &b) {
    // the FP32 copies of the centres (a NaN fails every comparison)
    return fabsf(b.xf) < 1e9f && fabsf(b.yf) < 1e9f && fabsf(b.xnf) < 1e9f &&
           fabsf(b.ynf) < 1e9f && b.r2f > 0.f && b.r2f < 1e12f;
}


// (i - X)^2 + (j - Y)^2 <= r^2, each operation rounded once (no contraction)
__device__ __forceinline__ bool inside_disk(int i, int j, double X, double Y, double r) {
    double dx = __dsub_rn((double)i, X), dy = __dsub_rn((double)j, Y);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= __dmul_rn(r, r);
}

// Map node coordinates into the domain; false beyond a non-periodic edge.
__device__ __forceinline__ bool locate(const Lattice &L, int x, int y, int &xo, int &yo) {
    if (L.bc_x == LBM_PERIODIC) {
        x %= L.nx;
        if (x < 0) x += L.nx;
    } else if (x < 0 || x >= L.nx) {
        return false;
    }
    if (L.bc_y == LBM_PERIODIC) {
        y %= L.ny;
        if (y < 0) y += L.ny;
    } else if (y < 0 || y >= L.ny) {
        return false;
    }
    xo = x;
    yo = y;
    return true;
}

// Inside test of node (i, j) for the disk (X, Y, r), decided exactly as the
// FP64 expression (i - X)^2 + (j - Y)^2 <= r^2.  An FP32 evaluation relative to
// the integer part of the centre settles every node farther than a relative
// 1e-5 from the circle; the rest use the FP64 expression itself.
struct DiskTest {
    double X, Y, r;
    int xi, yi;
    float fx, fy, r2, margin;
    // from a centre already split (split_coord) and the solid's r2f, rmf
    __device__ __forceinline__ DiskTest(double X_, double Y_, double r_, int xi_, int yi_,
                                        float fx_, float fy_, float r2_, float margin_)
        : X(X_), Y(Y_), r(r_), xi(xi_), yi(yi_), fx(fx_), fy(fy_), r2(r2_), margin(margin_) {}
    __device__ __forceinline__ DiskTest(double X_, double Y_, double r_) : X(X_), Y(Y_), r(r_) {
        const double fxd = floor(X), fyd = floor(Y);
        xi = (int)fxd;
        yi = (int)fyd;
        fx = (float)(X - fxd);
        fy = (float)(Y - fyd);
        r2 = (float)(r * r);
        margin = 1e-5f * r2 + 1e-5f;
    }
    __device__ __forceinline__ bool operator()(int i, int j) const {
        const float dx = (float)(i - xi) - fx, dy = (float)(j - yi) - fy;
        const float d2 = dx * dx + dy * dy;
        if (d2 < r2 - margin) return true;
        if (d2 > r2 + margin) return false;
        return inside_disk(i, j, X, Y, r);
    }
};

__device__ __forceinline__ void atomic_min_u16(uint16_t *a, uint16_t v) {
    unsigned short old = *reinterpret_cast<volatile unsigned short *>(a);
    while (v < old) {
        unsigned short seen = atomicCAS(reinterpret_cast<unsigned short *>(a), old, v);
        if (seen == old) break;
        old = seen;
    }
}

// Separation reduced to the nearest periodic image.
__device__ __forceinline__ double min_image(double d, int n, bool periodic) {
    if (!periodic) return d;
    double q = floor(__dadd_rn(__ddiv_rn(d, (double)n), 0.5));
    return __dsub_rn(d, __dmul_rn((double)n, q));
}

// Velocity V + Omega x (p - R) of a solid at the point p; d = p - R.
__device__ __forceinline__ void point_velocity(const Lattice &L, const double X, const double Y,
                                               double vx, double vy, double om, double px,
                                               double py, double &ux, double &uy, double &dx,
                                               double &dy) {
    dx = min_image(__dsub_rn(px, X), L.nx, L.bc_x == LBM_PERIODIC);
    dy = min_image(__dsub_rn(py, Y), L.ny, L.bc_y == LBM_PERIODIC);
    ux = vx - om * dy;
    uy = vy + om * dx;
}

// Interpolated boundary (the disks' boundary condition of the paper's
// simulations, ref. [40]): fraction q in (0, 1] of the link from the fluid
// node (x, y) along e_i at which it meets the circle of disk b, the smaller
// root of |p + q e_i - R|^2 = r^2 with p - R at the nearest periodic image.
__device__ __forceinline__ double link_fraction(const Lattice &L, const DSolid &b, int x, int y,
                                                int i) {
    const double px = min_image(__dsub_rn((double)x, b.x), L.nx, L.bc_x == LBM_PERIODIC);
    const double py = min_image(__dsub_rn((double)y, b.y), L.ny, L.bc_y == LBM_PERIODIC);
    const double ex = cx(i), ey = cy(i);
    const double a = ex * ex + ey * ey, h = px * ex + py * ey;
    const double cc = px * px + py * py - b.r * b.r;  // > 0: the node is outside
    const double disc = h * h - a * cc;
    double q = disc > 0.0 ? (-h - sqrt(disc)) / a : 0.5;
    if (!(q > 0.0)) q = 0.0;
    if (q > 1.0) q = 1.0;
    return q;
}

// The same fraction for the FP32 kernels, from the node's offset from the
// centre split as an integer part minus an FP32 remainder, (di - fx, dj - fy),
// along (ex, ey): the offset and c = |p - R|^2 - r^2 in FP64 without a
// division (the offset is exact, c to rounding), the root in FP32 by the
// conjugate form q = c / (-h + sqrt(h^2 - a c)), which loses no digits when
// the node lies close to the circle.  GB300 runs FP64 division and square
// root at a small fraction of its FP32 rate; these are the only ones this
// replaces.
__device__ __forceinline__ float link_fraction_split(int di, int dj, float fx, float fy, double r,
                                                     int ex, int ey) {
    const double px = (double)di - (double)fx, py = (double)dj - (double)fy;
    const double c = fma(px, px, fma(py, py, -r * r));  // > 0: the node is outside
    const float a = (float)(ex * ex + ey * ey), h = (float)(px * ex + py * ey);
    const float cf = (float)c, disc = h * h - a * cf;
    float q = 0.5f;
    if (disc > 0.f) {
        const float den = -h + sqrtf(disc);
        q = den > 0.f ? cf / den : 0.f;
    }
    if (!(q > 0.f)) q = 0.f;
    if (q > 1.f) q = 1.f;
    return q;
}

__device__ __forceinline__ long long cell_of(const Lattice &L, int x, int y) {
    return (long long)y * L.pitch + x;
}

// ----------------------------------------------------------- launchers

// Device tables of a batch of independent domains (k_stream_collide.cu and
// k_solid_step.cu).
struct BatchLaunch {
    StepParams *cases;        // [ncase], device; f0 = populations of the case's time t
    int4 *tiles;              // active tiles {case, x block, row, 0}, device
    int *ntiles;              // device
    int2 *items;              // active (case, local solid) pairs, device
    int *nitems;              // device
    int *active;              // active case ids, device
    int *nactive;             // device
    unsigned int *ticket;     // last-block ticket of the batch force kernel, device
    int precision, variant;
    bool force, local;
    int max_items;            // capacity of items (all solids of all cases)
    int max_tiles;            // tiles of all cases at the current tile shape
    int tile_h;               // rows per tile
    bool persistent;          // fused kernel: persistent blocks, else one block per tile
};

// Per-case convergence bookkeeping of a batch (device arrays of ncase).
struct BatchState {
    int ncase;
    double tol;
    long long max_steps;
    int *state;               // 0 active, 1 converged, 2 step cap, 3 unstable
    double *drag;             // drag at the previous test (NaN: none yet)
    int window;               // tests in a row within tol of the first that retire a case
    int *calm;                // tests in a row within tol of the anchor so far
    double *anchor;           // drag at the start of the current run of calm tests
    long long *steps;         // step counter of each case at the last test
    int *toff, *ioff;         // offsets of each active case in the tile and item lists
};

// k_stream_collide.cu
// the fused advection-collision kernel, and with variants 3-5 the pass over
// the nodes it leaves to the per-node update
constexpr int KERNEL_VARIANTS = 6;
inline bool deferred_path(const StepParams &p) {
    return p.collision != LBM_MRT && (p.sc_variant >= 3 || p.boundary == LBM_INTERPOLATED);
}
inline int stream_collide_launches(const StepParams &p) {
    return deferred_path(p) ? 2 : 1;  // MRT keeps the slow nodes inline
}
cudaError_t launch_stream_collide(const StepParams &p, cudaStream_t st);
// the update of the deferred per-node path, when list_by_forces
cudaError_t launch_deferred_update(const StepParams &p, cudaStream_t st);
// open channel: columns 0 and nx-1 of the populations just written (t+1)
cudaError_t launch_open_columns(const StepParams &p, cudaStream_t st);

// k_stream_collide_batch.cu
cudaError_t launch_stream_collide_batch(const BatchLaunch &b, cudaStream_t st);
int tile_nodes(int precision, int variant);  // nodes along x of one tile
// k_solid_step.cu: per-solid work of a step t -> t+1.  launch_forces: force
// record of time t and motion t -> t+1 of every solid; launch_ring after it:
// near lists when due, the moving solids' owner changes and covered/fresh
// nodes, listed (both only read what the advection-collision kernel of the
// step reads and write nothing it reads, so they may run beside it);
// launch_remask, after all three: the owner changes applied, refill, t += 1
// (one cooperative launch).
cudaError_t launch_forces(const StepParams &p, cudaStream_t st);
cudaError_t launch_ring(const StepParams &p, cudaStream_t st);
cudaError_t launch_remask(const StepParams &p, cudaStream_t st);
// batch: force record of every resting solid of every active case, t += 1
cudaError_t launch_solids_batch(const BatchLaunch &b, cudaStream_t st);
// batch: BATCH_TEST retires the active cases whose drag (Eq. 5 Fx summed
// over the case's solids) moved by less than tol relative since the previous
// test, or that reached max_steps or became unstable, and rebuilds the active
// case, item and tile lists when any case retired; BATCH_REBUILD clears the
// drag history and rebuilds the lists; BATCH_GATHER copies the step counters
// (all modes do).
constexpr int BATCH_TEST = 0, BATCH_REBUILD = 1, BATCH_GATHER = 2;
cudaError_t launch_batch_converge(const BatchLaunch &b, const BatchState &s, int mode,
                                  cudaStream_t st);

// k_solids.cu
cudaError_t launch_tick(const StepParams &p, cudaStream_t st);
cudaError_t launch_init_populations(const StepParams &p, cudaStream_t st);
cudaError_t launch_flags_all(const StepParams &p, cudaStream_t st);
cudaError_t launch_stamp_solid(const StepParams &p, int id, cudaStream_t st);
cudaError_t launch_export_populations(const StepParams &p, double *out, cudaStream_t st);
cudaError_t launch_import_populations(const StepParams &p, const double *in, cudaStream_t st);
cudaError_t launch_warm_start(const StepParams &p, const float *pred, double u_scale,
                              double rho_scale, int base, cudaStream_t st);
cudaError_t launch_export_owner(const StepParams &p, int32_t *out, cudaStream_t st);
cudaError_t launch_case_features(const StepParams &p, double re, float *in, cudaStream_t st);
cudaError_t launch_fields(const StepParams &p, double *rho, double *ux, double *uy,
                          cudaStream_t st);
cudaError_t launch_link_masks(const StepParams &p, uint8_t *mask, cudaStream_t st);

}  // namespace gbm
