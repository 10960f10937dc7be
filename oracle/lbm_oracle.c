/*
 * Plain FP64 CPU oracle for the D2Q9 lattice-Boltzmann step with moving rigid
 * disks, half-way bounce-back, fresh/covered node handling and the two
 * momentum-exchange force evaluations of Wen, Zhang, Tu, Wang and Fang,
 * "Galilean Invariant Fluid-Solid Interfacial Dynamics in Lattice Boltzmann
 * Simulations" (arXiv:1303.0625).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of the method that the CUDA library is checked against.  Only the
 * test-suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it; the CUDA library never calls it and shares no code,
 * header or table with it.
 *
 * Everything is double precision, written as loops in the order the paper
 * states the method.  Built with OpenMP, the two per-node loops (advection
 * with bounce-back, collision) are shared among threads; every node's result
 * depends only on the previous state, so the output does not depend on the
 * thread count.  Sums over links, node-type changes and solids stay serial.  Compile with floating-point contraction disabled
 * (-ffp-contract=off) so that the geometric inside tests are rounded exactly
 * as written.
 *
 * One step t -> t+1 is, in this order:
 *   1. forces at t on every solid from every fluid-solid link: the
 *      conventional form (Eq. 4) and the Galilean-invariant form (Eq. 5),
 *      summed into total force (Eq. 6) and torque (Eq. 7), plus the momentum
 *      booked by the node-type changes of the previous step (Sec. I);
 *   2. advection (Eq. 3) in pull form; a population whose source node is
 *      solid (or a channel wall) is the half-way bounced-back population with
 *      the moving-wall term (Sec. III.A);
 *   3. BGK collision (Eq. 2) towards the equilibrium of Eq. 8;
 *   4. solid motion (prescribed, or Newton-Euler driven by the Eq. 5 force);
 *   5. re-rasterisation of the solids: nodes a solid moves over ("covered")
 *      give their momentum to it, nodes it uncovers ("fresh", newborn) are
 *      refilled by extrapolation along the surrounding fluid-solid links
 *      (Sec. IV.B, algorithm A1, averaged over the participating links) and
 *      take their momentum from it.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - weights 4/9, 1/9, 1/36 (the only D2Q9 weights for which Eq. 10 holds);
 *   - BGK: Omega = -(f - feq)/tau;
 *   - moving-wall term of the bounced population: +6 w_i rho_w (e_i . v),
 *     with rho_w either rho0 or the local density of the fluid node;
 *   - the intersection point of a half-way link: x_s = x_f + e_i / 2;
 *   - v at a point p of a solid: V + Omega x (p - R);
 *   - a node is inside a disk iff (i-X)^2 + (j-Y)^2 <= r^2, lowest solid id
 *     wins where disks overlap;
 *   - covered node: +rho u of its post-collision populations; fresh node:
 *     -rho u of its refilled populations; torque about R(t+1);
 *   - refill: A1 = 3 f(x+e) - 3 f(x+2e) + f(x+3e) along every direction whose
 *     three nodes are old fluid; else A2 = 2 f(x+e) - f(x+2e); else A3 =
 *     neighbour average; else equilibrium at rho0 and the solid velocity;
 *   - open channel (bc_x = ORA_OPEN, not part of the paper's method): after
 *     collision the inlet column x = 0 and the outlet column x = nx-1 take the
 *     non-equilibrium extrapolation of their inner neighbour n (x = 1 and
 *     x = nx-2): f_b = feq(rho_b, u_b) + (f_n - feq(rho_n, u_n)), with f_n
 *     post-collision and rho_n, u_n its moments; the inlet imposes the
 *     parabolic velocity u_b = (u_in(y), 0) with rho_b = rho_n, the outlet
 *     the density rho_b = rho0 with u_b = u_n.  Where the neighbour is solid
 *     the inlet is feq(rho0, u_in) and the outlet updates as a node whose
 *     outside neighbours are a resting wall.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 discrete velocities in the order printed in Sec. III.C. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* index of the opposite velocity, e_opp(i) = -e_i */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* weighting coefficients of Eq. 8 (not printed in the paper; see above) */
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

#define ORA_PI 3.14159265358979323846

#define ORA_PERIODIC 0
#define ORA_WALL 1
#define ORA_OPEN 2 /* x only: Poiseuille velocity inlet at x=0, pressure outlet at x=nx-1 */

#define ORA_PRESCRIBED 0
#define ORA_FREE 1

typedef struct {
    int32_t nx, ny;
    int32_t bc_x, bc_y;
    double tau;
    double rho0;
    double u0x, u0y;       /* initial uniform velocity */
    double wall_ux[2];     /* x-velocity of the y=-1/2 wall [0] and the y=ny-1/2 wall [1] */
    double body_fx, body_fy; /* uniform body force on the fluid (Guo forcing) */
    double inflow_umax;    /* peak of the Poiseuille inlet profile (bc_x = ORA_OPEN) */
    double gravity_x, gravity_y; /* gravity on free solids */
    double lub_range;      /* gap below which the repulsive lubrication force acts */
    int32_t rho_w_mode;    /* 0: rho_w = rho0; 1: rho_w = density of the fluid node */
    int32_t refill;        /* 1: A1, 2: A2, 3: A3 */
    int32_t motion_cme;    /* 1: free solids move under Eq. 4; 0: under Eq. 5 */
    int32_t relative_changes; /* 1: the Eq. 5 record books a covered or fresh node's
                               * momentum relative to the boundary, m (u - v) */
    int32_t collision;     /* 0: BGK; 1: MRT with the rates of Sec. IV (no body force) */
    int32_t boundary;      /* disks: 0 half-way bounce-back; 1 interpolated (ref. [40]) */
} ora_config;

typedef struct {
    double xa, ya;   /* position when added (prescribed motion starts from it) */
    int64_t ta;      /* time when added */
    double x, y;     /* centre of mass R(t) */
    double vx, vy;   /* velocity V(t) */
    double om;       /* angular velocity Omega(t) */
    double r, rho_s;
    int32_t motion;
} ora_solid;

typedef struct {
    ora_config c;
    int64_t t;
    int nsolid, cap;
    ora_solid *s;
    double *f;        /* post-collision populations at time t, [9][ny][nx] */
    double *g;        /* populations after advection, before collision */
    int32_t *owner;   /* -1 fluid, else id of the solid covering the node */
    int32_t *owner_prev;
    uint8_t *fresh;
    double *pending;  /* [nsolid][3] momentum booked for the next force record */
    double *pending_rel; /* [nsolid][3] the same, relative to the boundary velocity */
    int raster_dirty; /* solids added since the owner map was last built */
} ora_sim;

/* ------------------------------------------------------------------ basics */

static size_t cells(const ora_sim *S) { return (size_t)S->c.nx * (size_t)S->c.ny; }
static size_t at(const ora_sim *S, int x, int y) { return (size_t)y * S->c.nx + x; }
static double *F(const ora_sim *S, double *base, int i, int x, int y)
{
    return base + (size_t)i * cells(S) + at(S, x, y);
}

static int wrap(int i, int n)
{
    i %= n;
    if (i < 0) i += n;
    return i;
}

/* Map node coordinates into the domain.  Returns 0 when the node lies beyond
 * a non-periodic boundary. */
static int locate(const ora_sim *S, int x, int y, int *xo, int *yo)
{
    if (S->c.bc_x == ORA_PERIODIC) x = wrap(x, S->c.nx);
    else if (x < 0 || x >= S->c.nx) return 0;
    if (S->c.bc_y == ORA_PERIODIC) y = wrap(y, S->c.ny);
    else if (y < 0 || y >= S->c.ny) return 0;
    *xo = x;
    *yo = y;
    return 1;
}

/* Separation along one axis, reduced to the nearest periodic image. */
static double min_image(double d, int n, int periodic)
{
    if (!periodic) return d;
    return d - (double)n * floor(d / (double)n + 0.5);
}

/* Eq. 8: equilibrium distribution. */
void ora_feq(double rho, double ux, double uy, double *out)
{
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; i++) {
        double eu = EX[i] * ux + EY[i] * uy;
        out[i] = rho * W[i] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Velocity of solid s at the point (px, py): V + Omega x (p - R). */
static void solid_point_velocity(const ora_sim *S, int s, double px, double py, double *vx,
                                 double *vy, double *dx, double *dy)
{
    const ora_solid *b = &S->s[s];
    double ddx = min_image(px - b->x, S->c.nx, S->c.bc_x == ORA_PERIODIC);
    double ddy = min_image(py - b->y, S->c.ny, S->c.bc_y == ORA_PERIODIC);
    *vx = b->vx - b->om * ddy;
    *vy = b->vy + b->om * ddx;
    *dx = ddx;
    *dy = ddy;
}

static double local_density(const ora_sim *S, const double *f, int x, int y)
{
    double rho = 0.0;
    for (int j = 0; j < 9; j++) rho += *F(S, (double *)f, j, x, y);
    return rho;
}

/*
 * Force on a solid from one fluid-solid link (x_f, i), x_f + e_i inside the
 * solid.  fi = f~_i(x_f, t) streams into the boundary; fbb = f~_opp(x_b, t)
 * streams out of it, i.e. the bounced-back population that arrives at x_f.
 * out[0..1] = Eq. 4 (conventional), out[2..3] = Eq. 5 (Galilean invariant,
 * relative velocities e_i - v and e_opp - v).
 */
void ora_link_force(int i, double fi, double fbb, double vx, double vy, double *out)
{
    int o = OPP[i];
    out[0] = EX[i] * fi - EX[o] * fbb;
    out[1] = EY[i] * fi - EY[o] * fbb;
    out[2] = (EX[i] - vx) * fi - (EX[o] - vx) * fbb;
    out[3] = (EY[i] - vy) * fi - (EY[o] - vy) * fbb;
}

/* Half-way bounce-back with the moving-wall term: the population leaving
 * x_f along e_i returns along e_opp carrying  f~_i - 6 w_i rho_w (e_i . v). */
static double bounced(int i, double fi, double rho_w, double vx, double vy)
{
    return fi - 6.0 * W[i] * rho_w * (EX[i] * vx + EY[i] * vy);
}

/* --------------------------------------------- interpolated boundary
 * The boundary condition the paper's simulations use (Sec. IV, ref. [40]):
 * the disk's surface cuts a link at its true position, at fraction q of the
 * link from the fluid node, instead of half-way, and the returning population
 * is interpolated linearly from the populations near the wall.  The channel
 * walls stay half-way (they lie at y = -1/2 and ny - 1/2). */

/* Fraction q in (0, 1] of the link from the fluid node (x, y) along e_i at
 * which it meets the circle of solid s (the node lies outside, x + e_i
 * inside): the smaller root of |p + q e_i - R|^2 = r^2, with p - R at the
 * nearest periodic image. */
static double link_fraction(const ora_sim *S, int s, int x, int y, int i)
{
    const ora_solid *b = &S->s[s];
    double px = min_image((double)x - b->x, S->c.nx, S->c.bc_x == ORA_PERIODIC);
    double py = min_image((double)y - b->y, S->c.ny, S->c.bc_y == ORA_PERIODIC);
    double a = (double)(EX[i] * EX[i] + EY[i] * EY[i]);
    double h = px * EX[i] + py * EY[i];
    double cc = px * px + py * py - b->r * b->r; /* > 0: the node is outside */
    double disc = h * h - a * cc;
    double q = disc > 0.0 ? (-h - sqrt(disc)) / a : 0.5;
    if (!(q > 0.0)) q = 0.0;
    if (q > 1.0) q = 1.0;
    return q;
}

/* Population i arriving at the fluid node (x, y) from solid s, whose surface
 * cuts the link along e_opp(i) at fraction q, from the post-collision
 * populations f:
 *   q < 1/2:  2q f_opp(x) + (1 - 2q) f_opp(x + e_i) + M
 *   q >= 1/2: (f_opp(x) + M) / (2q) + (2q - 1) / (2q) f_i(x)
 * with the moving-wall term M = 6 w_i rho_w (e_i . v), v the solid's velocity
 * at the cut x - q e_i.  q = 1/2 is the half-way rule; where x + e_i is not a
 * fluid node of the domain the half-way value f_opp(x) + M is taken.  Returns
 * the cut's velocity and its offset from the centre through v and d. */
static double returning(const ora_sim *S, double *f, int x, int y, int i, int s, double rho_w,
                        double *vx, double *vy, double *dx, double *dy)
{
    const int o = OPP[i];
    const double q = link_fraction(S, s, x, y, o);
    solid_point_velocity(S, s, (double)x - q * EX[i], (double)y - q * EY[i], vx, vy, dx, dy);
    const double back = *F(S, f, o, x, y);
    const double m = 6.0 * W[i] * rho_w * (EX[i] * *vx + EY[i] * *vy);
    if (q >= 0.5) return (back + m) / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * *F(S, f, i, x, y);
    int xn, yn;
    if (!locate(S, x + EX[i], y + EY[i], &xn, &yn) || S->owner[at(S, xn, yn)] >= 0)
        return back + m;
    return 2.0 * q * back + (1.0 - 2.0 * q) * *F(S, f, o, xn, yn) + m;
}

/* -------------------------------------------------------- rasterisation */

static int inside_disk(double px, double py, double X, double Y, double r)
{
    double dx = px - X, dy = py - Y;
    return dx * dx + dy * dy <= r * r;
}

/* owner map of all solids at their current centres: lowest id wins. */
static void rasterise(const ora_sim *S, int32_t *owner)
{
    for (size_t k = 0; k < cells(S); k++) owner[k] = -1;
    for (int s = 0; s < S->nsolid; s++) {
        const ora_solid *b = &S->s[s];
        int x0 = (int)floor(b->x - b->r), x1 = (int)ceil(b->x + b->r);
        int y0 = (int)floor(b->y - b->r), y1 = (int)ceil(b->y + b->r);
        for (int j = y0; j <= y1; j++)
            for (int i = x0; i <= x1; i++) {
                int xi, yi;
                if (!inside_disk((double)i, (double)j, b->x, b->y, b->r)) continue;
                if (!locate(S, i, j, &xi, &yi)) continue;
                if (owner[at(S, xi, yi)] < 0) owner[at(S, xi, yi)] = s;
            }
    }
}

/* ---------------------------------------------------------------- set-up */

static double inlet_ux(const ora_config *c, int y)
{
    double h = (double)c->ny;
    double yy = (double)y + 0.5;
    return 4.0 * c->inflow_umax * yy * (h - yy) / (h * h);
}

ora_sim *ora_create(const ora_config *c)
{
    if (c->nx < 4 || c->ny < 4 || !(c->tau > 0.5)) return NULL;
    if (c->motion_cme != 0 && c->motion_cme != 1) return NULL;
    if (c->relative_changes != 0 && c->relative_changes != 1) return NULL;
    if (c->collision != 0 && c->collision != 1) return NULL;
    if (c->collision == 1 && (c->body_fx != 0.0 || c->body_fy != 0.0)) return NULL;
    if (c->boundary != 0 && c->boundary != 1) return NULL;
    ora_sim *S = (ora_sim *)calloc(1, sizeof(ora_sim));
    S->c = *c;
    S->cap = 16;
    S->s = (ora_solid *)calloc((size_t)S->cap, sizeof(ora_solid));
    S->pending = (double *)calloc((size_t)S->cap * 3, sizeof(double));
    S->pending_rel = (double *)calloc((size_t)S->cap * 3, sizeof(double));
    S->f = (double *)calloc(9 * cells(S), sizeof(double));
    S->g = (double *)calloc(9 * cells(S), sizeof(double));
    S->owner = (int32_t *)malloc(cells(S) * sizeof(int32_t));
    S->owner_prev = (int32_t *)malloc(cells(S) * sizeof(int32_t));
    S->fresh = (uint8_t *)calloc(cells(S), 1);
    for (size_t k = 0; k < cells(S); k++) S->owner[k] = S->owner_prev[k] = -1;
    /* f~(0) = feq(rho0, u0); the open channel starts from the inlet profile */
    for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++) {
            double e[9];
            double ux = c->bc_x == ORA_OPEN ? inlet_ux(c, y) : c->u0x;
            double uy = c->bc_x == ORA_OPEN ? 0.0 : c->u0y;
            ora_feq(c->rho0, ux, uy, e);
            for (int i = 0; i < 9; i++) *F(S, S->f, i, x, y) = e[i];
        }
    return S;
}

void ora_destroy(ora_sim *S)
{
    if (!S) return;
    free(S->s);
    free(S->pending);
    free(S->pending_rel);
    free(S->f);
    free(S->g);
    free(S->owner);
    free(S->owner_prev);
    free(S->fresh);
    free(S);
}

int ora_add_disk(ora_sim *S, double cx, double cy, double r, double vx, double vy, double om,
                 double rho_s, int motion)
{
    if (S->nsolid == S->cap) {
        S->cap *= 2;
        S->s = (ora_solid *)realloc(S->s, (size_t)S->cap * sizeof(ora_solid));
        S->pending = (double *)realloc(S->pending, (size_t)S->cap * 3 * sizeof(double));
        S->pending_rel = (double *)realloc(S->pending_rel, (size_t)S->cap * 3 * sizeof(double));
    }
    int id = S->nsolid++;
    ora_solid *b = &S->s[id];
    b->xa = b->x = cx;
    b->ya = b->y = cy;
    b->ta = S->t;
    b->vx = vx;
    b->vy = vy;
    b->om = om;
    b->r = r;
    b->rho_s = rho_s;
    b->motion = motion;
    S->pending[3 * id] = S->pending[3 * id + 1] = S->pending[3 * id + 2] = 0.0;
    S->pending_rel[3 * id] = S->pending_rel[3 * id + 1] = S->pending_rel[3 * id + 2] = 0.0;
    S->raster_dirty = 1; /* rasterised before the owner map is next used */
    return id;
}

/* Owner map of the current solids (added solids cover their nodes without
 * booking any momentum). */
static void ensure_raster(ora_sim *S)
{
    if (!S->raster_dirty) return;
    rasterise(S, S->owner);
    memcpy(S->owner_prev, S->owner, cells(S) * sizeof(int32_t));
    S->raster_dirty = 0;
}

/* ------------------------------------------------------- 1. forces at t */

/* rec: [nsolid][2][3] = {conventional, Galilean} x {Fx, Fy, T}. */
static void record_forces(ora_sim *S, double *rec)
{
    const ora_config *c = &S->c;
    memset(rec, 0, (size_t)S->nsolid * 6 * sizeof(double));
    for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++) {
            if (S->owner[at(S, x, y)] >= 0) continue;
            double rho_w = c->rho_w_mode ? local_density(S, S->f, x, y) : c->rho0;
            for (int i = 1; i < 9; i++) {
                int xb, yb;
                if (!locate(S, x + EX[i], y + EY[i], &xb, &yb)) continue;
                int s = S->owner[at(S, xb, yb)];
                if (s < 0) continue;
                double vx, vy, dx, dy, fbb;
                double fi = *F(S, S->f, i, x, y);
                if (c->boundary) {
                    /* the population that returns to x along e_opp(i), and the
                     * velocity and lever arm at the cut */
                    fbb = returning(S, S->f, x, y, OPP[i], s, rho_w, &vx, &vy, &dx, &dy);
                } else {
                    /* intersection point of the half-way link */
                    double xs = (double)x + 0.5 * EX[i], ys = (double)y + 0.5 * EY[i];
                    solid_point_velocity(S, s, xs, ys, &vx, &vy, &dx, &dy);
                    fbb = bounced(i, fi, rho_w, vx, vy);
                }
                double lf[4];
                ora_link_force(i, fi, fbb, vx, vy, lf);
                double *r = rec + 6 * s;
                r[0] += lf[0];                   /* Eq. 6 */
                r[1] += lf[1];
                r[2] += dx * lf[1] - dy * lf[0]; /* Eq. 7 */
                r[3] += lf[2];
                r[4] += lf[3];
                r[5] += dx * lf[3] - dy * lf[2];
            }
        }
    for (int s = 0; s < S->nsolid; s++) {
        double *r = rec + 6 * s, *p = S->pending + 3 * s, *q = S->pending_rel + 3 * s;
        const double *pg = S->c.relative_changes ? q : p; /* what the Eq. 5 record books */
        r[0] += p[0];
        r[1] += p[1];
        r[2] += p[2];
        r[3] += pg[0];
        r[4] += pg[1];
        r[5] += pg[2];
        p[0] = p[1] = p[2] = 0.0;
        q[0] = q[1] = q[2] = 0.0;
    }
}

/* ------------------------------------------------- 2. advection (pull) */

static void advect(ora_sim *S)
{
    const ora_config *c = &S->c;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++) {
            if (S->owner[at(S, x, y)] >= 0) {
                for (int i = 0; i < 9; i++) *F(S, S->g, i, x, y) = 0.0;
                continue;
            }
            double rho_w = c->rho_w_mode ? local_density(S, S->f, x, y) : c->rho0;
            for (int i = 0; i < 9; i++) {
                int sx = x - EX[i], sy = y - EY[i];
                double back = *F(S, S->f, OPP[i], x, y);
                double val;
                if (c->bc_y == ORA_WALL && (sy < 0 || sy >= c->ny)) {
                    /* channel wall at y = -1/2 or y = ny - 1/2, moving along x.
                     * The population leaving x along e_opp returns along e_i. */
                    double uw = c->wall_ux[sy < 0 ? 0 : 1];
                    val = bounced(OPP[i], back, rho_w, uw, 0.0);
                } else if (c->bc_x != ORA_PERIODIC && (sx < 0 || sx >= c->nx)) {
                    /* resting wall at x = -1/2 or x = nx - 1/2 (an open column
                     * is overwritten after collision) */
                    val = back;
                } else {
                    int xs, ys;
                    locate(S, sx, sy, &xs, &ys);
                    int s = S->owner[at(S, xs, ys)];
                    if (s >= 0 && c->boundary) {
                        double vx, vy, dx, dy;
                        val = returning(S, S->f, x, y, i, s, rho_w, &vx, &vy, &dx, &dy);
                    } else if (s >= 0) {
                        double vx, vy, dx, dy;
                        solid_point_velocity(S, s, (double)x - 0.5 * EX[i], (double)y - 0.5 * EY[i],
                                             &vx, &vy, &dx, &dy);
                        val = bounced(OPP[i], back, rho_w, vx, vy);
                    } else {
                        val = *F(S, S->f, i, xs, ys);
                    }
                }
                *F(S, S->g, i, x, y) = val;
            }
        }
}

/* ------------------------------------------------------ 3. collision */

/* Open column x = b from its inner neighbour x = n (both fluid), after the
 * neighbour's collision: non-equilibrium extrapolation.  The neighbour's
 * density and velocity are those of its collision (pre-collision moments,
 * half the body force in u).  inlet: velocity (u_in(y), 0) with the
 * neighbour's density; outlet: density rho0 with the neighbour's velocity. */
static void open_column(ora_sim *S, int b, int n, int y, int inlet)
{
    const ora_config *c = &S->c;
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; i++) {
        double g = *F(S, S->g, i, n, y);
        rho += g;
        jx += EX[i] * g;
        jy += EY[i] * g;
    }
    double ux = (jx + 0.5 * c->body_fx) / rho, uy = (jy + 0.5 * c->body_fy) / rho;
    double eq_n[9], eq_b[9];
    ora_feq(rho, ux, uy, eq_n);
    if (inlet) ora_feq(rho, inlet_ux(c, y), 0.0, eq_b);
    else ora_feq(c->rho0, ux, uy, eq_b);
    for (int i = 0; i < 9; i++)
        *F(S, S->f, i, b, y) = eq_b[i] + (*F(S, S->f, i, n, y) - eq_n[i]);
}

/* ---------------------------------------------------------------- MRT
 * Multiple-relaxation-time collision (Sec. IV names it, with the rates
 * S = diag(0, 1.64, 1.54, 0, 1.9, 0, 1.9, 1/tau, 1/tau)): moments m = M f in
 * the basis (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy) of the D2Q9 model of
 * the paper's refs. [33, 45], each moment relaxed at its rate towards the
 * moment of the equilibrium Eq. 8, m_eq = M f_eq, then f = M^-1 m.  Row k of M
 * evaluates a polynomial in (e_x, e_y) at the nine velocities; M^-1 is
 * obtained by Gauss-Jordan elimination. */
static double MRT_M[9][9], MRT_MI[9][9];
static int mrt_ready = 0;

static void mrt_init(void)
{
    if (mrt_ready) return;
    for (int i = 0; i < 9; i++) {
        double ex = EX[i], ey = EY[i], e2 = ex * ex + ey * ey;
        MRT_M[0][i] = 1.0;                                   /* rho */
        MRT_M[1][i] = 3.0 * e2 - 4.0;                        /* e: energy */
        MRT_M[2][i] = 4.5 * e2 * e2 - 10.5 * e2 + 4.0;       /* eps: energy squared */
        MRT_M[3][i] = ex;                                    /* j_x */
        MRT_M[4][i] = (3.0 * e2 - 5.0) * ex;                 /* q_x: energy flux */
        MRT_M[5][i] = ey;                                    /* j_y */
        MRT_M[6][i] = (3.0 * e2 - 5.0) * ey;                 /* q_y */
        MRT_M[7][i] = ex * ex - ey * ey;                     /* p_xx: normal stress */
        MRT_M[8][i] = ex * ey;                               /* p_xy: shear stress */
    }
    double a[9][18];
    for (int r = 0; r < 9; r++)
        for (int k = 0; k < 18; k++) a[r][k] = k < 9 ? MRT_M[r][k] : (k - 9 == r ? 1.0 : 0.0);
    for (int col = 0; col < 9; col++) {
        int piv = col;
        for (int r = col + 1; r < 9; r++)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        for (int k = 0; k < 18; k++) {
            double tmp = a[col][k];
            a[col][k] = a[piv][k];
            a[piv][k] = tmp;
        }
        double d = a[col][col];
        for (int k = 0; k < 18; k++) a[col][k] /= d;
        for (int r = 0; r < 9; r++) {
            if (r == col || a[r][col] == 0.0) continue;
            double m = a[r][col];
            for (int k = 0; k < 18; k++) a[r][k] -= m * a[col][k];
        }
    }
    for (int r = 0; r < 9; r++)
        for (int k = 0; k < 9; k++) MRT_MI[r][k] = a[r][9 + k];
    mrt_ready = 1;
}

/* One MRT collision of the populations f of a node with rates s[9]. */
void ora_mrt_node(const double *f, const double *s, double *out)
{
    mrt_init();
    double rho = 0.0, jx = 0.0, jy = 0.0, eq[9], m[9], meq[9], ms[9];
    for (int i = 0; i < 9; i++) {
        rho += f[i];
        jx += EX[i] * f[i];
        jy += EY[i] * f[i];
    }
    ora_feq(rho, jx / rho, jy / rho, eq);
    for (int k = 0; k < 9; k++) {
        m[k] = meq[k] = 0.0;
        for (int i = 0; i < 9; i++) {
            m[k] += MRT_M[k][i] * f[i];
            meq[k] += MRT_M[k][i] * eq[i];
        }
        ms[k] = m[k] - s[k] * (m[k] - meq[k]);
    }
    for (int i = 0; i < 9; i++) {
        out[i] = 0.0;
        for (int k = 0; k < 9; k++) out[i] += MRT_MI[i][k] * ms[k];
    }
}

/* The rates of Sec. IV: conserved moments 0, e 1.64, eps 1.54, q 1.9, stress 1/tau. */
static void mrt_rates(double tau, double *s)
{
    const double r[9] = {0.0, 1.64, 1.54, 0.0, 1.9, 0.0, 1.9, 1.0 / tau, 1.0 / tau};
    for (int k = 0; k < 9; k++) s[k] = r[k];
}

static void collide(ora_sim *S)
{
    const ora_config *c = &S->c;
    double tau = c->tau, Fx = c->body_fx, Fy = c->body_fy;
    if (c->collision == 1) mrt_init(); /* before the threads share the tables */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++) {
            if (S->owner[at(S, x, y)] >= 0) {
                for (int i = 0; i < 9; i++) *F(S, S->f, i, x, y) = 0.0;
                continue;
            }
            double g[9], rho = 0.0, jx = 0.0, jy = 0.0;
            for (int i = 0; i < 9; i++) {
                g[i] = *F(S, S->g, i, x, y);
                rho += g[i];
                jx += EX[i] * g[i];
                jy += EY[i] * g[i];
            }
            if (c->collision == 1) {
                double s[9], out[9];
                mrt_rates(tau, s);
                ora_mrt_node(g, s, out);
                for (int i = 0; i < 9; i++) *F(S, S->f, i, x, y) = out[i];
                continue;
            }
            /* Guo forcing: u includes half the body force */
            double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
            double eq[9];
            ora_feq(rho, ux, uy, eq);
            for (int i = 0; i < 9; i++) {
                double eu = EX[i] * ux + EY[i] * uy;
                double src = (1.0 - 0.5 / tau) * W[i] *
                             (3.0 * ((EX[i] - ux) * Fx + (EY[i] - uy) * Fy) +
                              9.0 * eu * (EX[i] * Fx + EY[i] * Fy));
                *F(S, S->f, i, x, y) = g[i] - (g[i] - eq[i]) / tau + src;
            }
        }
    if (c->bc_x == ORA_OPEN) {
        for (int y = 0; y < c->ny; y++) {
            double eq[9];
            if (S->owner[at(S, 0, y)] < 0) {
                if (S->owner[at(S, 1, y)] < 0) {
                    open_column(S, 0, 1, y, 1);
                } else {
                    ora_feq(c->rho0, inlet_ux(c, y), 0.0, eq);
                    for (int i = 0; i < 9; i++) *F(S, S->f, i, 0, y) = eq[i];
                }
            }
            if (S->owner[at(S, c->nx - 1, y)] < 0 && S->owner[at(S, c->nx - 2, y)] < 0)
                open_column(S, c->nx - 1, c->nx - 2, y, 0);
        }
    }
}

/* -------------------------------------------------------- 4. motion */

/* Repulsive force on disk a from disk b (or a wall) when their gap is below
 * the range zeta:  kappa ((zeta - gap) / zeta)^2 along the unit normal. */
static double lub_mag(double kappa, double zeta, double gap)
{
    if (gap >= zeta) return 0.0;
    double q = (zeta - gap) / zeta;
    return kappa * q * q;
}

static double net_weight(const ora_sim *S, const ora_solid *b)
{
    double M = b->rho_s * ORA_PI * b->r * b->r;
    double g = sqrt(S->c.gravity_x * S->c.gravity_x + S->c.gravity_y * S->c.gravity_y);
    return fabs(1.0 - S->c.rho0 / b->rho_s) * M * g;
}

static void move_solids(ora_sim *S, const double *rec)
{
    const ora_config *c = &S->c;
    int n = S->nsolid;
    double *fl = (double *)calloc((size_t)n * 2 + 2, sizeof(double));
    /* pairwise lubrication between free solids and walls */
    for (int a = 0; a < n; a++) {
        const ora_solid *A = &S->s[a];
        if (A->motion != ORA_FREE || !(c->lub_range > 0.0)) continue;
        double ka = net_weight(S, A);
        for (int b = 0; b < n; b++) {
            if (b == a) continue;
            const ora_solid *B = &S->s[b];
            double dx = min_image(A->x - B->x, c->nx, c->bc_x == ORA_PERIODIC);
            double dy = min_image(A->y - B->y, c->ny, c->bc_y == ORA_PERIODIC);
            double d = sqrt(dx * dx + dy * dy);
            double kb = net_weight(S, B);
            double m = lub_mag(ka > kb ? ka : kb, c->lub_range, d - A->r - B->r);
            if (m > 0.0 && d > 0.0) {
                fl[2 * a] += m * dx / d;
                fl[2 * a + 1] += m * dy / d;
            }
        }
        if (c->bc_y == ORA_WALL) {
            fl[2 * a + 1] += lub_mag(ka, c->lub_range, (A->y - A->r) + 0.5);
            fl[2 * a + 1] -= lub_mag(ka, c->lub_range, ((double)c->ny - 0.5) - (A->y + A->r));
        }
        if (c->bc_x == ORA_WALL) {
            fl[2 * a] += lub_mag(ka, c->lub_range, (A->x - A->r) + 0.5);
            fl[2 * a] -= lub_mag(ka, c->lub_range, ((double)c->nx - 0.5) - (A->x + A->r));
        }
    }
    for (int s = 0; s < n; s++) {
        ora_solid *b = &S->s[s];
        if (b->motion == ORA_PRESCRIBED) {
            double dt = (double)(S->t + 1 - b->ta);
            b->x = b->xa + b->vx * dt;
            b->y = b->ya + b->vy * dt;
            continue;
        }
        /* Newton-Euler in FP64 driven by the Galilean-invariant force (Eq. 5),
         * or by the conventional one (Eq. 4) when the configuration asks */
        double M = b->rho_s * ORA_PI * b->r * b->r;
        double I = 0.5 * M * b->r * b->r;
        double buoy = 1.0 - c->rho0 / b->rho_s;
        const double *r = rec + 6 * s + (c->motion_cme ? 0 : 3);
        double Fx = r[0] + buoy * M * c->gravity_x + fl[2 * s];
        double Fy = r[1] + buoy * M * c->gravity_y + fl[2 * s + 1];
        double vx1 = b->vx + Fx / M, vy1 = b->vy + Fy / M;
        b->x += 0.5 * (b->vx + vx1);
        b->y += 0.5 * (b->vy + vy1);
        b->vx = vx1;
        b->vy = vy1;
        b->om += r[2] / I;
    }
    free(fl);
}

/* --------------------------------------------- 5. node-type changes */

/* A node that may feed a refill: inside the domain, fluid, not newborn. */
static int usable(const ora_sim *S, int x, int y, size_t *k)
{
    int xi, yi;
    if (!locate(S, x, y, &xi, &yi)) return 0;
    *k = at(S, xi, yi);
    return S->owner[*k] < 0 && !S->fresh[*k];
}

/* Populations for a newborn fluid node (x, y) uncovered by solid s. */
static void refill_node(ora_sim *S, int x, int y, int s, double *out)
{
    const size_t N = cells(S);
    int mode = S->c.refill;
    double acc[9];
    int count;
    size_t k1, k2, k3;
    if (mode <= 1) { /* A1: second-order extrapolation along each link */
        count = 0;
        memset(acc, 0, sizeof acc);
        for (int i = 1; i < 9; i++) {
            if (!usable(S, x + EX[i], y + EY[i], &k1)) continue;
            if (!usable(S, x + 2 * EX[i], y + 2 * EY[i], &k2)) continue;
            if (!usable(S, x + 3 * EX[i], y + 3 * EY[i], &k3)) continue;
            for (int j = 0; j < 9; j++)
                acc[j] += 3.0 * S->f[j * N + k1] - 3.0 * S->f[j * N + k2] + S->f[j * N + k3];
            count++;
        }
        if (count) {
            for (int j = 0; j < 9; j++) out[j] = acc[j] / count;
            return;
        }
    }
    if (mode <= 2) { /* A2: linear extrapolation */
        count = 0;
        memset(acc, 0, sizeof acc);
        for (int i = 1; i < 9; i++) {
            if (!usable(S, x + EX[i], y + EY[i], &k1)) continue;
            if (!usable(S, x + 2 * EX[i], y + 2 * EY[i], &k2)) continue;
            for (int j = 0; j < 9; j++) acc[j] += 2.0 * S->f[j * N + k1] - S->f[j * N + k2];
            count++;
        }
        if (count) {
            for (int j = 0; j < 9; j++) out[j] = acc[j] / count;
            return;
        }
    }
    /* A3: average of the neighbouring fluid nodes */
    count = 0;
    memset(acc, 0, sizeof acc);
    for (int i = 1; i < 9; i++) {
        if (!usable(S, x + EX[i], y + EY[i], &k1)) continue;
        for (int j = 0; j < 9; j++) acc[j] += S->f[j * N + k1];
        count++;
    }
    if (count) {
        for (int j = 0; j < 9; j++) out[j] = acc[j] / count;
        return;
    }
    double vx = 0.0, vy = 0.0, dx, dy;
    if (s >= 0) solid_point_velocity(S, s, (double)x, (double)y, &vx, &vy, &dx, &dy);
    ora_feq(S->c.rho0, vx, vy, out);
}

static void remask(ora_sim *S)
{
    const ora_config *c = &S->c;
    const size_t N = cells(S);
    memcpy(S->owner_prev, S->owner, N * sizeof(int32_t));
    rasterise(S, S->owner);
    memset(S->fresh, 0, N);
    for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++) {
            size_t k = at(S, x, y);
            int was = S->owner_prev[k], now = S->owner[k];
            if (was < 0 && now >= 0) {
                /* covered: the node's momentum goes to the solid; relative to
                 * the boundary it is m (u - v), m the node's mass */
                double jx = 0.0, jy = 0.0, m = 0.0, vx, vy, dx, dy;
                for (int j = 0; j < 9; j++) {
                    jx += EX[j] * S->f[j * N + k];
                    jy += EY[j] * S->f[j * N + k];
                    m += S->f[j * N + k];
                }
                solid_point_velocity(S, now, (double)x, (double)y, &vx, &vy, &dx, &dy);
                double *p = S->pending + 3 * now, *q = S->pending_rel + 3 * now;
                p[0] += jx;
                p[1] += jy;
                p[2] += dx * jy - dy * jx;
                const double rx = jx - m * vx, ry = jy - m * vy;
                q[0] += rx;
                q[1] += ry;
                q[2] += dx * ry - dy * rx;
            }
            if (was >= 0 && now < 0) S->fresh[k] = 1;
        }
    for (int y = 0; y < c->ny; y++)
        for (int x = 0; x < c->nx; x++) {
            size_t k = at(S, x, y);
            if (!S->fresh[k]) continue;
            int s = S->owner_prev[k];
            double nf[9], jx = 0.0, jy = 0.0, m = 0.0, vx, vy, dx, dy;
            refill_node(S, x, y, s, nf);
            for (int j = 0; j < 9; j++) {
                S->f[j * N + k] = nf[j];
                jx += EX[j] * nf[j];
                jy += EY[j] * nf[j];
                m += nf[j];
            }
            /* newborn: the solid gives the node its momentum (relative: m (u - v)) */
            solid_point_velocity(S, s, (double)x, (double)y, &vx, &vy, &dx, &dy);
            double *p = S->pending + 3 * s, *q = S->pending_rel + 3 * s;
            p[0] -= jx;
            p[1] -= jy;
            p[2] -= dx * jy - dy * jx;
            const double rx = jx - m * vx, ry = jy - m * vy;
            q[0] -= rx;
            q[1] -= ry;
            q[2] -= dx * ry - dy * rx;
        }
}

/* ------------------------------------------------------------ one step */

/* Advance n steps.  rec (may be NULL) receives [n][nsolid][2][3]. */
void ora_step(ora_sim *S, int64_t n, double *rec)
{
    double *r = (double *)malloc(((size_t)S->nsolid * 6 + 1) * sizeof(double));
    ensure_raster(S);
    for (int64_t k = 0; k < n; k++) {
        record_forces(S, r);
        if (rec) memcpy(rec + (size_t)k * S->nsolid * 6, r, (size_t)S->nsolid * 6 * sizeof(double));
        advect(S);
        collide(S);
        move_solids(S, r);
        remask(S);
        S->t++;
    }
    free(r);
}

/* --------------------------------------------------------- accessors */

/* Fraction of the link from (x, y) along e_i at which it meets solid s. */
double ora_link_fraction(const ora_sim *S, int s, int x, int y, int i)
{
    return link_fraction(S, s, x, y, i);
}

/* Threads of the per-node loops (1 without OpenMP); n < 1 selects all cores. */
int ora_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n >= 1 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int64_t ora_time(const ora_sim *S) { return S->t; }
int ora_nsolid(const ora_sim *S) { return S->nsolid; }

void ora_get_f(const ora_sim *S, double *out) { memcpy(out, S->f, 9 * cells(S) * sizeof(double)); }
void ora_set_f(ora_sim *S, const double *in) { memcpy(S->f, in, 9 * cells(S) * sizeof(double)); }
void ora_get_owner(ora_sim *S, int32_t *out)
{
    ensure_raster(S);
    memcpy(out, S->owner, cells(S) * sizeof(int32_t));
}

/* density and velocity of the post-collision state; solid nodes get NaN.
 * With a body force the velocity is (sum e f~ - F/2) / rho. */
void ora_fields(ora_sim *S, double *rho, double *ux, double *uy)
{
    const size_t N = cells(S);
    ensure_raster(S);
    for (size_t k = 0; k < N; k++) {
        if (S->owner[k] >= 0) {
            rho[k] = ux[k] = uy[k] = NAN;
            continue;
        }
        double r = 0.0, jx = 0.0, jy = 0.0;
        for (int j = 0; j < 9; j++) {
            r += S->f[j * N + k];
            jx += EX[j] * S->f[j * N + k];
            jy += EY[j] * S->f[j * N + k];
        }
        rho[k] = r;
        ux[k] = (jx - 0.5 * S->c.body_fx) / r;
        uy[k] = (jy - 0.5 * S->c.body_fy) / r;
    }
}

/* [x, y, vx, vy, omega] of solid s */
void ora_solid_state(const ora_sim *S, int s, double *out)
{
    const ora_solid *b = &S->s[s];
    out[0] = b->x;
    out[1] = b->y;
    out[2] = b->vx;
    out[3] = b->vy;
    out[4] = b->om;
}

void ora_set_solid_state(ora_sim *S, int s, const double *in)
{
    ora_solid *b = &S->s[s];
    b->x = in[0];
    b->y = in[1];
    b->vx = in[2];
    b->vy = in[3];
    b->om = in[4];
    /* prescribed motion restarts from here */
    b->xa = b->x;
    b->ya = b->y;
    b->ta = S->t;
}

/* Enumerate the fluid-solid links in raster order of the fluid node and
 * ascending direction.  Writes up to cap entries of (x_f, y_f, i, solid). */
int64_t ora_links(ora_sim *S, int64_t cap, int32_t *out)
{
    int64_t n = 0;
    ensure_raster(S);
    for (int y = 0; y < S->c.ny; y++)
        for (int x = 0; x < S->c.nx; x++) {
            if (S->owner[at(S, x, y)] >= 0) continue;
            for (int i = 1; i < 9; i++) {
                int xb, yb;
                if (!locate(S, x + EX[i], y + EY[i], &xb, &yb)) continue;
                int s = S->owner[at(S, xb, yb)];
                if (s < 0) continue;
                if (n < cap) {
                    out[4 * n] = x;
                    out[4 * n + 1] = y;
                    out[4 * n + 2] = i;
                    out[4 * n + 3] = s;
                }
                n++;
            }
        }
    return n;
}

/* Refill value the newborn node (x, y) would get if it alone were fresh,
 * uncovered by solid s, given the current populations and owner map. */
void ora_refill_probe(ora_sim *S, int x, int y, int s, double *out)
{
    ensure_raster(S);
    memset(S->fresh, 0, cells(S));
    S->fresh[at(S, x, y)] = 1;
    refill_node(S, x, y, s, out);
    S->fresh[at(S, x, y)] = 0;
}

/* Momentum [nsolid][3] booked by the last node-type changes, which the next
 * force record will carry. */
void ora_pending(const ora_sim *S, double *out)
{
    memcpy(out, S->pending, (size_t)S->nsolid * 3 * sizeof(double));
}
