/*
 * lbm.h - C ABI of the GB300 library for the D2Q9 lattice-Boltzmann step with
 * moving rigid disks and the Galilean-invariant momentum-exchange force of
 * Wen, Zhang, Tu, Wang and Fang, arXiv:1303.0625.
 *
 * The library owns every device buffer it allocates (populations, owner map,
 * node flags, solid table, force history).  The caller owns every output
 * buffer it passes in.  All entry points return an lbm_status and never abort
 * or exit.  A context is not thread-safe; separate contexts are independent.
 *
 * Lattice conventions (Sec. III.C of the paper):
 *   velocities e_0..e_8 = (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1),
 *   weights 4/9 (i=0), 1/9 (i=1..4), 1/36 (i=5..8);
 *   node (x, y) sits at integer coordinates, 0 <= x < nx, 0 <= y < ny;
 *   every 2-D field is row-major [ny][nx] (x fastest); populations are
 *   [9][ny][nx].
 * One step t -> t+1 (Eq. 1-3) records the force on every solid at t (Eq. 4-7
 * plus the momentum of nodes that changed type), advects with half-way
 * bounce-back, collides (BGK, Eq. 2 and Eq. 8), moves the solids and
 * re-rasterises them (covered nodes give their momentum to the solid, fresh
 * nodes are refilled by extrapolation, Sec. IV.B).
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque; owns all device state */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,    /* bad argument or configuration; nothing changed */
    LBM_ENOMEM = 2,    /* a device or host allocation failed */
    LBM_ECUDA = 3,     /* a CUDA call failed; lbm_last_error has the text */
    LBM_EUNSTABLE = 4, /* a non-finite or non-positive density was produced */
    LBM_ETIMEOUT = 5,  /* a bounded device wait ran out */
    LBM_ESTATE = 6,    /* call not valid in the current state (e.g. record gone) */
} lbm_status;

/* boundary kinds for bc_x / bc_y */
enum {
    LBM_PERIODIC = 0,
    LBM_WALL = 1, /* half-way bounce-back wall half a spacing outside the first/last node */
    LBM_OPEN = 2, /* x only: parabolic velocity inlet column x=0 (peak inflow_umax), pressure
                   * outlet column x=nx-1 (density rho0), both by non-equilibrium
                   * extrapolation from the inner neighbour column */
};
/* storage / arithmetic precision */
enum {
    LBM_FP64 = 0,     /* populations stored and computed in FP64 */
    LBM_FP32_DEV = 1, /* stored as f_i - w_i in FP32, computed in FP32 */
    LBM_FP16_DEV = 2, /* stored as f_i - w_i in FP16, computed in FP32 */
};
/* density used in the moving-wall term of the bounced population */
enum { LBM_RHOW_CONST = 0 /* rho0 */, LBM_RHOW_LOCAL = 1 /* density of the fluid node */ };
/* newborn-node refill (Sec. IV.B): A1 2nd-order, A2 linear, A3 neighbour average */
enum { LBM_REFILL_A1 = 1, LBM_REFILL_A2 = 2, LBM_REFILL_A3 = 3 };
/* solid motion */
enum { LBM_PRESCRIBED = 0, LBM_FREE = 1 };
/* collision model: BGK (single relaxation time, Eq. 2) or MRT with the rates of
 * Sec. IV, S = diag(0, 1.64, 1.54, 0, 1.9, 0, 1.9, 1/tau, 1/tau) on the moments
 * (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy); MRT takes no body force and
 * runs one launch shape (lbm_set_kernel_variant has no effect on it) */
enum { LBM_BGK = 0, LBM_MRT = 1 };
/* boundary condition on the disks: half-way bounce-back with the moving-wall
 * term (Sec. III.A), or the interpolated boundary of the paper's simulations
 * (Sec. IV, ref. [40]): the surface cuts the link from a fluid node x at
 * fraction q (from the circle), and the returned population is
 *   q <  1/2: 2q f~_opp(x) + (1 - 2q) f~_opp(x + e_i) + M
 *   q >= 1/2: (f~_opp(x) + M) / (2q) + (2q - 1) / (2q) f~_i(x)
 * with M = 6 w_i rho_w (e_i . v) and v the disk's velocity at the cut (the
 * half-way value where x + e_i is not a fluid node).  The Eq. 4/5 forces use
 * the same returned population, and v and the torque lever at the cut.  The
 * channel walls stay half-way.  With it, BGK runs the per-node path in the
 * deferred pass (kernel variants 0-2 act as 3-5).  Batches take LBM_HALFWAY
 * only. */
enum { LBM_HALFWAY = 0, LBM_INTERPOLATED = 1 };
/* force form: Eq. 4 (conventional) or Eq. 5 (Galilean invariant) */
enum { LBM_CME = 0, LBM_GME = 1 };

typedef struct {
    int32_t nx, ny;        /* nodes; 4 <= nx, ny and nx * ny < 2^31 */
    int32_t bc_x, bc_y;    /* LBM_PERIODIC | LBM_WALL | LBM_OPEN (x only) */
    double tau;            /* BGK relaxation time (> 0.5); viscosity (tau - 1/2) / 3 */
    double rho0;           /* initial density and rho_w in LBM_RHOW_CONST */
    double u0[2];          /* initial uniform velocity (ignored when bc_x = LBM_OPEN) */
    double wall_ux[2];     /* x-velocity of the y = -1/2 wall [0] and y = ny-1/2 wall [1] */
    double body_force[2];  /* uniform body force on the fluid (Guo forcing); 0 = none */
    double inflow_umax;    /* peak of the parabolic inlet profile for bc_x = LBM_OPEN */
    double gravity[2];     /* gravity acting on free solids (net of buoyancy) */
    double lub_range;      /* gap below which free solids repel; 0 = off */
    int32_t precision;     /* LBM_FP64 | LBM_FP32_DEV | LBM_FP16_DEV */
    int32_t rho_w_mode;    /* LBM_RHOW_CONST | LBM_RHOW_LOCAL */
    int32_t refill;        /* LBM_REFILL_A1 (default) | A2 | A3 */
    int32_t force_ring;    /* number of most recent steps whose forces stay on device (>= 1) */
    int32_t device;        /* CUDA device ordinal */
    int32_t motion_cme;    /* force driving LBM_FREE solids: 0 = Eq. 5 (Galilean invariant,
                            * default), 1 = Eq. 4 (conventional; for comparison) */
    int32_t relative_changes; /* momentum of covered/fresh nodes in the Eq. 5 record:
                               * 0 = m u as in the Eq. 4 record (default), 1 = m (u - v)
                               * relative to the boundary velocity v at the node */
    int32_t collision;     /* LBM_BGK (default) | LBM_MRT; batches take LBM_BGK only */
    int32_t boundary;      /* disks: LBM_HALFWAY (default) | LBM_INTERPOLATED */
    void *stream;          /* cudaStream_t to run on; NULL = a stream the context creates */
} lbm_config;

typedef struct {
    double cx, cy;   /* centre R at the current time, lattice units */
    double r;        /* radius; nodes with (x-cx)^2 + (y-cy)^2 <= r^2 are solid */
    double vx, vy;   /* translational velocity V */
    double omega;    /* angular velocity (counter-clockwise positive) */
    double rho_s;    /* solid density (used by LBM_FREE motion) */
    int32_t motion;  /* LBM_PRESCRIBED: R(t) = R_add + V (t - t_add); LBM_FREE: Newton-Euler */
    int32_t reserved;/* must be 0 */
} lbm_disk;

/* Fill *cfg with defaults: periodic 64x64, tau 0.8, rho0 1, FP32_DEV,
 * RHOW_CONST, REFILL_A1, force_ring 256, device 0, own stream. */
void lbm_config_default(lbm_config *cfg);

/* Create a context: allocate the populations (two buffers), owner map, node
 * flags and force history on cfg->device and set every population to the
 * equilibrium of Eq. 8 at (rho0, u0) (the inlet profile for an open channel).
 * On success *out owns the device memory until lbm_destroy.
 * Errors: LBM_EINVAL (tau <= 0.5, sizes, enum values, reserved != 0),
 * LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_create(const lbm_config *cfg, lbm_ctx **out);

/* Release everything the context owns.  NULL is accepted. */
lbm_status lbm_destroy(lbm_ctx *ctx);

/* Add a rigid disk at the current time and rasterise it into the owner map
 * (nodes it covers become solid; no momentum is booked for them).  The solid
 * is the moving boundary of Sec. III.A: a rigid body whose surface point S
 * has the velocity v = V + Omega x (S - R) that enters the bounced population
 * and Eq. 5; LBM_FREE disks are the freely moving cylinders of Sec. IV
 * (translation and rotation under gravity and the hydrodynamic force of
 * Eq. 6-7).  Solid ids
 * are 0, 1, ... in order of addition; where disks overlap the lowest id owns
 * the node.  Errors: LBM_EINVAL (r <= 0, r >= min(nx, ny) / 2 - 4, centre not
 * finite, rho_s <= 0 for a free disk, more than 65534 solids). */
lbm_status lbm_add_solid(lbm_ctx *ctx, const lbm_disk *disk, int32_t *id_out);

/* Enqueue nsteps steps on the context's stream; returns without waiting.
 * One step t -> t+1 is the lattice Boltzmann equation Eq. 1 split into
 * collision Eq. 2 (BGK towards Eq. 8) and advection Eq. 3, with the solids'
 * links handled by bounce-back and the moving-wall term (Sec. III.A), the
 * force record of time t by Eq. 4-7 before advection, the solids' motion,
 * and the node-type changes of Sec. I (covered nodes' momentum to the solid,
 * fresh nodes refilled by the extrapolation of Sec. IV.B).
 * Device errors from earlier work surface here or at the next call that
 * waits.  nsteps >= 0. */
lbm_status lbm_step(lbm_ctx *ctx, int64_t nsteps);

/* Wait for all enqueued work.  The status a step's kernels raised:
 * LBM_EUNSTABLE for a non-finite or non-positive density or a non-finite
 * solid state; LBM_ETIMEOUT when a grid barrier of the per-solid kernel gave
 * up; LBM_ESTATE when a solid covered or uncovered more than 256 nodes in one
 * step (its event queue), the step's owner changes overflowed their list
 * (twice the event lists' room), or the deferred list of nodes next to
 * solids overflowed (the step's momentum booking, re-rasterisation or
 * slow-node update is then incomplete).  These conditions persist: every later waiting call returns
 * them until lbm_load restores a saved state. */
lbm_status lbm_sync(lbm_ctx *ctx);

/* Copy the force records of steps first_step .. first_step+count-1 into out,
 * laid out [count][nsolid][3] = (Fx, Fy, T) of the chosen form (Eq. 4 or
 * Eq. 5, each summed by Eq. 6 and Eq. 7, plus the covered/fresh node
 * momenta).  The record of step t is the force at time t, taken before the
 * step t -> t+1 advects.  Records exist for the last force_ring steps taken;
 * asking for older or future ones gives LBM_ESTATE.  on_device != 0: out is a
 * device pointer and the copy is enqueued on the context's stream; otherwise
 * out is host memory and the call waits. */
lbm_status lbm_forces(lbm_ctx *ctx, int32_t form, int64_t first_step, int64_t count, double *out,
                      int32_t on_device);

/* Density and velocity of the current post-collision state, each [ny][nx]
 * FP64: the moments of Sec. II, rho = sum_i f_i and rho u = sum_i e_i f_i
 * (collision conserves both, so pre- and post-collision agree); solid nodes
 * are NaN.  With a body force the velocity is (sum_i e_i f_i - F/2) / rho.
 * on_device as for lbm_forces. */
lbm_status lbm_fields(lbm_ctx *ctx, double *rho, double *ux, double *uy, int32_t on_device);

/* Same result as lbm_fields(ctx, rho, ux, uy, 0), for callers that must not
 * allocate device memory.  The paper has no counterpart: this is a service of
 * the library.  A program whose device memory is held by another allocator
 * (PyTorch's caching allocator keeps freed blocks for itself, so a plain
 * cudaMalloc can fail although the process has memory to spare), or which must
 * not stall other streams (cudaFree waits for the whole device), cannot afford
 * the staging buffer that lbm_fields allocates on first use.  This entry point
 * stages the three fields in one fixed array compiled into the library
 * instead (LBM_FIELDS_STATIC_MAX_NODES nodes, 3 doubles each, 12 MiB reserved
 * on every GPU that loads the library, until the process exits).
 * rho, ux, uy: host arrays [ny][nx]; solid nodes are NaN.  Waits for the
 * stream.  Errors: LBM_EINVAL for a NULL argument or nx * ny above the
 * maximum (nothing is copied then).  The first call on a device looks up the
 * array's device address, so make that first call before any stream capture.
 * Every call uses the same array and it keeps the last call's contents;
 * calls whose work overlaps on the GPU (two contexts on different streams of
 * one device, or several threads) race on it and must be serialised. */
#define LBM_FIELDS_STATIC_MAX_NODES 524288
lbm_status lbm_fields_static(lbm_ctx *ctx, double *rho, double *ux, double *uy);

/* Current populations as FP64 [9][ny][nx] (converted from the storage
 * precision; the values at solid nodes are unspecified) / overwrite them
 * (rounded to the storage precision).  on_device as for lbm_forces. */
lbm_status lbm_get_populations(lbm_ctx *ctx, double *f, int32_t on_device);
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f, int32_t on_device);

/* Checkpoints.  A saved state holds everything the next steps depend on: the
 * populations of the current time in the storage precision, the owner map,
 * the node flags, the solid table (FP64 centres, velocities, closed-form
 * motion origins), the force history, the momenta the last re-rasterisation
 * booked into the next force record, and the step counter.  lbm_state_size
 * gives the bytes lbm_save needs now (they change with the step's
 * covered/fresh event count).  lbm_save waits for the stream, then copies the
 * state into buf (host memory the caller owns); it returns the status of the
 * steps taken (a state after LBM_EUNSTABLE or LBM_ETIMEOUT is not saved).
 * lbm_load restores a state into a context created with the same
 * configuration (stream and device aside) and holding the same solids (the
 * same lbm_add_solid calls): the status word and the bounded waits' counters
 * are cleared, and the steps that follow give the same results, bit for bit,
 * as those that followed the save.  Errors: LBM_EINVAL for a buffer that is
 * too small, not a saved state, or from another configuration or solid
 * count (nothing is changed then); a batch's cases are not saved one by
 * one.  This is a service of the library; the paper has none. */
lbm_status lbm_state_size(lbm_ctx *ctx, int64_t *bytes);
lbm_status lbm_save(lbm_ctx *ctx, void *buf, int64_t bytes);
lbm_status lbm_load(lbm_ctx *ctx, const void *buf, int64_t bytes);

/* Owner map [ny][nx]: -1 for fluid, else the id of the solid covering the
 * node.  on_device as for lbm_forces. */
lbm_status lbm_get_owner(lbm_ctx *ctx, int32_t *owner, int32_t on_device);

/* Solid state at the current time, host [nsolid][5] = (x, y, vx, vy, omega).
 * Waits for the stream. */
lbm_status lbm_get_solids(lbm_ctx *ctx, double *state);

/* Set the velocity and angular velocity of solid id.  state = (x, y, vx,
 * vy, omega) where (x, y) must equal the current centre exactly (positions
 * cannot be changed; LBM_EINVAL otherwise).  A prescribed disk restarts its
 * closed-form motion R(t) = R + V (t - now) from its current centre. */
lbm_status lbm_set_solid(lbm_ctx *ctx, int32_t id, const double *state);

/* Fluid-solid links (x_f fluid, x_f + e_i solid, Eq. 6 summation set) as
 * host rows (x_f, y_f, i, solid) in raster order of x_f then ascending i.
 * Writes min(cap, total) rows and stores the total in *n_out. Waits. */
lbm_status lbm_links(lbm_ctx *ctx, int64_t cap, int32_t *out, int64_t *n_out);

/* Current time step and number of solids. */
int64_t lbm_time(const lbm_ctx *ctx);
int32_t lbm_nsolid(const lbm_ctx *ctx);

/* Human-readable text of the last error on ctx (or of the last failed
 * lbm_create when ctx is NULL).  Owned by the library. */
const char *lbm_last_error(const lbm_ctx *ctx);
const char *lbm_status_string(lbm_status st);

/* Bounded device waits: a grid-wide barrier of the re-rasterisation kernel
 * gives up after `polls` polls of about 64 ns (default 2^24, about one
 * second); the launch then stops, and the next call that waits returns
 * LBM_ETIMEOUT (the step's per-solid work is incomplete: restore a state
 * saved by lbm_save before stepping on).  0 gives up at once, so that every
 * step with moving solids times out: the time-out path can be exercised
 * without a stalled device.  LBM_EINVAL for polls < 0. */
lbm_status lbm_set_wait_limit(lbm_ctx *ctx, int64_t polls);

/* Launch policy.  steps_per_graph > 1 captures that many steps into one CUDA
 * graph and replays it; 0 or 1 launches each kernel directly (default 0). */
lbm_status lbm_set_graph(lbm_ctx *ctx, int32_t steps_per_graph);

/* Kernel timing: while enabled, every launch of the fused advection-collision
 * kernel is bracketed by CUDA events on the context's stream (graphs are not
 * used).  lbm_get_timing waits, then returns the summed duration in ms and the
 * number of launches since timing was enabled. */
lbm_status lbm_set_timing(lbm_ctx *ctx, int32_t enable);
lbm_status lbm_get_timing(lbm_ctx *ctx, double *stream_collide_ms, int64_t *launches);

/* Kernel launches issued by the library since creation (all kernels). */
int64_t lbm_launch_count(const lbm_ctx *ctx);

/* Launch variant of the advection-collision kernel.  Nodes per thread, as
 * the width of one population word: 0 = 16 bytes (default), 1 = 8 bytes,
 * 2 = 4 bytes; 3, 4, 5 = the same widths with the nodes next to solids and
 * edges (the per-node path) computed by a second kernel after the first
 * instead of inline.  Every variant evaluates the same expressions; the
 * compiler may fuse multiply-adds differently in each, so results agree to
 * the storage precision's rounding (not always bit for bit).  LBM_EINVAL for
 * other values. */
lbm_status lbm_set_kernel_variant(lbm_ctx *ctx, int32_t variant);
int32_t lbm_kernel_variant(const lbm_ctx *ctx);

/* Where the force kernel of a step (force record of time t, motion) runs:
 * 1 = on a second stream of the context, beside the advection-collision
 * kernel, which reads the same state (default); 0 = before it, on the
 * context's stream.  Results do not depend on it.  LBM_EINVAL for other
 * values. */
lbm_status lbm_set_force_overlap(lbm_ctx *ctx, int32_t on);
int32_t lbm_force_overlap(const lbm_ctx *ctx);

/* Autotuner: run 1 + steps real steps with each of the 6 variants of the
 * advection-collision kernel, with the force kernel beside it and before it,
 * timing whole steps with CUDA events, and keep the fastest pair (the variant
 * stored in *best when not NULL; lbm_force_overlap tells the other).  The
 * simulation advances by 12 (1 + steps) steps; results do not depend on the
 * choice.  Waits for the stream. */
lbm_status lbm_autotune(lbm_ctx *ctx, int32_t steps, int32_t *best);

/* ------------------------------------------------------------------ batches
 *
 * A batch runs many independent domains ("cases", e.g. a sweep of channels
 * with one fixed cylinder each) as one set of launches per step: one
 * advection-collision launch over the tiles of every active case, one launch
 * for the force records of every solid of every active case, and every
 * `every` steps one launch that tests convergence and retires cases.  The
 * method is the paper's (Eq. 1-8) applied to each case on its own; batching
 * is an execution scheme the paper does not have.  Each case is an lbm_ctx
 * that the batch owns; its results are read through the lbm_ctx calls above.
 *
 * Limits: every case has the same precision, rho_w_mode and device; solids
 * in a batch rest (zero velocity, prescribed), so no node changes type. */
typedef struct lbm_batch lbm_batch; /* opaque; owns its cases */

/* case states */
enum {
    LBM_CASE_ACTIVE = 0,    /* still stepping */
    LBM_CASE_CONVERGED = 1, /* drag moved by less than tol (relative) over `every` steps */
    LBM_CASE_CAPPED = 2,    /* reached max_steps without converging */
    LBM_CASE_UNSTABLE = 3,  /* a status bit was raised or the drag became non-finite */
};

/* Create ncase cases from configs[0..ncase-1] (lbm_create's rules for each;
 * precision, rho_w_mode and device equal for all, else LBM_EINVAL).  The
 * batch runs on configs[0].stream (or a stream it creates); the other
 * configs' stream fields are ignored.  Convergence defaults: every = 100,
 * tol = 1e-7, max_steps = 2000000. */
lbm_status lbm_batch_create(const lbm_config *configs, int32_t ncase, lbm_batch **out);
lbm_status lbm_batch_destroy(lbm_batch *b);

/* Number of cases, and a borrowed handle of case k (valid until
 * lbm_batch_destroy).  Reading calls (lbm_forces, lbm_fields, lbm_time,
 * lbm_get_populations, lbm_get_owner, lbm_get_solids, lbm_links) and
 * lbm_set_populations work on it; calls that step it or change its solids
 * return LBM_EINVAL (use the lbm_batch_* calls). */
int32_t lbm_batch_size(const lbm_batch *b);
lbm_status lbm_batch_case(lbm_batch *b, int32_t k, lbm_ctx **ctx);

/* Add a resting disk (vx = vy = omega = 0, LBM_PRESCRIBED; else LBM_EINVAL)
 * to case k; lbm_add_solid's rules otherwise.  Its id within the case is
 * stored in *id when not NULL. */
lbm_status lbm_batch_add_solid(lbm_batch *b, int32_t k, const lbm_disk *d, int32_t *id);

/* Convergence test: every `every` steps of the batch (>= 1), an active case
 * whose drag D (x component of the Eq. 5 force summed over its solids, from
 * its latest record) satisfies |D - D_prev| < tol |D|, D_prev being the drag
 * at the previous test, becomes LBM_CASE_CONVERGED and stops stepping; one
 * that has run max_steps steps becomes LBM_CASE_CAPPED.  A case without
 * solids has D = 0 and never converges.  The drag history restarts. */
lbm_status lbm_batch_set_convergence(lbm_batch *b, int32_t every, double tol, int64_t max_steps);

/* Number of tests in a row whose drag must stay within tol (relative) of the
 * drag at the test before them for a case to retire as converged (default 1:
 * the test as stated above).  A single test also passes at a turning point of
 * an oscillating drag, and in FP32 storage the drag's round-off noise (a few
 * 1e-7 per 100 steps) decides whether a tolerance below it ever passes; a
 * band held over many tests does neither.  The drag history restarts.
 * LBM_EINVAL for tests < 1. */
lbm_status lbm_batch_set_convergence_window(lbm_batch *b, int32_t tests);

/* Advance every active case by up to `steps` steps (fewer when all cases
 * retire first; the test runs whenever the batch has done `every` steps since
 * the previous one).  *nactive (when not NULL) receives the number of active
 * cases afterwards.  Waits for the stream. */
lbm_status lbm_batch_run(lbm_batch *b, int64_t steps, int32_t *nactive);

/* Per-case results after the last lbm_batch_run, host arrays of ncase (any
 * may be NULL): state (LBM_CASE_*), steps run, drag at the latest test (NaN
 * before the first). */
lbm_status lbm_batch_state(lbm_batch *b, int32_t *state, int64_t *steps, double *drag);

/* Retire the active cases ids[0..n-1] now (state LBM_CASE_CONVERGED): the
 * caller's own criterion was met.  Retired or out-of-range ids: LBM_EINVAL,
 * nothing changed.  The drag history restarts. */
lbm_status lbm_batch_retire(lbm_batch *b, const int32_t *ids, int32_t n);

/* Launch policy.  Tiles of the fused kernel are tile_rows rows (1..64) of
 * 128 threads x the nodes per thread of `variant` (as for
 * lbm_set_kernel_variant).  persistent = 1 runs the fused kernel as resident
 * blocks walking the tile list, 0 as one block per tile (default).  graph = 1
 * captures the `every` steps between two tests (and the test) into one CUDA
 * graph (default 1).  Defaults: variant 0, 1 row, per-tile blocks. */
lbm_status lbm_batch_set_launch(lbm_batch *b, int32_t variant, int32_t tile_rows,
                                int32_t persistent, int32_t graph);
lbm_status lbm_batch_get_launch(const lbm_batch *b, int32_t *variant, int32_t *tile_rows,
                                int32_t *persistent);

/* Autotuner: run 1 + steps real steps with each of LBM_BATCH_TUNE_SHAPES
 * launch shapes (variant, rows per tile, persistent), timing the fused
 * kernel with CUDA events, and keep the fastest (stored in best[0..2] when
 * not NULL).  The batch advances by LBM_BATCH_TUNE_SHAPES (1 + steps) steps
 * and the drag history restarts.  Waits for the stream. */
#define LBM_BATCH_TUNE_SHAPES 10
lbm_status lbm_batch_autotune(lbm_batch *b, int32_t steps, int32_t *best);

/* Timing of the fused kernel as for lbm_set_timing / lbm_get_timing. */
lbm_status lbm_batch_set_timing(lbm_batch *b, int32_t enable);
lbm_status lbm_batch_get_timing(lbm_batch *b, double *stream_collide_ms, int64_t *launches);

/* Kernel launches issued by the batch (all kernels), and the text of its
 * last error (owned by the library). */
int64_t lbm_batch_launch_count(const lbm_batch *b);
const char *lbm_batch_last_error(const lbm_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
