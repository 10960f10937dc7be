// Host side of the C ABI declared in include/lbm.h: context lifetime, solid
// table, step scheduling (direct launches or a captured CUDA graph), force
// history, field export and kernel timing.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <mutex>

#include "lbm_internal.cuh"
#include "lbm_nn.h"

using gbm::DSolid;
using gbm::StepParams;

struct lbm_ctx {
    lbm_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int pitch = 0;
    size_t elem = 0;
    void *f[2] = {nullptr, nullptr};
    uint16_t *owner = nullptr, *flags = nullptr;
    DSolid *solids = nullptr;
    int solid_cap = 0;
    int nsolid = 0;
    int *moving_d = nullptr;
    int moving_cap = 0;
    void *ev_d = nullptr;  // covered/fresh events: {length, pad}, int4 list, 6 doubles each
    int ev_cap = 0;
    int *bnd_d = nullptr;  // deferred per-node path: {length by step parity, list}
    int bnd_cap = 0;
    long long bnd_need = 0;  // sum over disks of their box sizes
    std::vector<int> moving;
    std::vector<uint8_t> is_moving;
    double *ring = nullptr;
    int ring_cap = 0;      // solids the ring was laid out for
    long long *t_d = nullptr;
    int *status_d = nullptr;
    unsigned int *bar_d = nullptr;  // per-solid control words (barrier, displacement, pair test)
    uint16_t *near_d = nullptr;     // near lists, [solid_cap][NEAR_CAP]
    long long spin_limit = 1ll << 24;  // polls of a bounded device wait (about one second)
    // the force kernel runs on a second stream beside the advection-collision
    // kernel: fork after the previous step, join before the re-rasterisation
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    bool overlap = true;  // force kernel beside the advection-collision kernel (else before it)
    int64_t t = 0;
    int64_t ring_base = 0; // first step whose force record is valid
    std::string err;
    // launch policy
    int graph_steps = 0;
    int sc_variant = 0;
    cudaGraphExec_t gexec = nullptr;
    // timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    double timed_ms = 0.0;
    int64_t timed_launches = 0;
    int64_t launches = 0;
    int64_t graph_launches = 0;  // kernel launches in one replay of gexec
    // staging buffer for host transfers
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    // set when the context is a case of a batch (stepped by the batch only)
    const lbm_batch *batch = nullptr;
};

namespace {

thread_local std::string g_create_error;

lbm_status fail(lbm_ctx *c, lbm_status st, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
lbm_status fail(lbm_ctx *c, lbm_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return st;
}

#define CK(ctx, call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,    \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                   \
    } while (0)

size_t elem_bytes(int prec) { return prec == LBM_FP64 ? 8 : (prec == LBM_FP32_DEV ? 4 : 2); }

StepParams params(const lbm_ctx *c) {
    StepParams p{};
    const lbm_config &g = c->cfg;
    p.L.nx = g.nx;
    p.L.ny = g.ny;
    p.L.pitch = c->pitch;
    p.L.bc_x = g.bc_x;
    p.L.bc_y = g.bc_y;
    p.L.plane = (long long)g.ny * c->pitch;
    p.f0 = c->f[0];
    p.f1 = c->f[1];
    p.owner = c->owner;
    p.flags = c->flags;
    p.S = c->solids;
    p.nsolid = c->nsolid;
    p.moving = c->moving_d;
    p.nmoving = (int)c->moving.size();
    p.ring = c->ring;
    p.ring_len = g.force_ring + 1;
    p.t = c->t_d;
    p.status = c->status_d;
    p.tau = g.tau;
    p.omega = 1.0 / g.tau;
    p.rho0 = g.rho0;
    p.wall_ux0 = g.wall_ux[0];
    p.wall_ux1 = g.wall_ux[1];
    p.body_x = g.body_force[0];
    p.body_y = g.body_force[1];
    p.umax = g.inflow_umax;
    p.grav_x = g.gravity[0];
    p.grav_y = g.gravity[1];
    p.lub = g.lub_range;
    p.u0x = g.u0[0];
    p.u0y = g.u0[1];
    p.rho_w_mode = g.rho_w_mode;
    p.refill = g.refill;
    p.motion_cme = g.motion_cme;
    p.relative_changes = g.relative_changes;
    p.collision = g.collision;
    p.boundary = g.boundary;
    p.precision = g.precision;
    p.sc_variant = c->sc_variant;
    p.bnd = c->bnd_d;
    p.bnd_cap = c->bnd_cap;
    // with solids on the deferred per-node path, the force kernel lists the
    // nodes next to them (it visits them anyway)
    p.list_by_forces = c->nsolid > 0 && c->bnd_d && gbm::deferred_path(p) ? 1 : 0;
    p.ev_len = static_cast<int *>(c->ev_d);
    p.ev = c->ev_d ? reinterpret_cast<int4 *>(static_cast<char *>(c->ev_d) + 16) : nullptr;
    p.ev_mom = c->ev_d ? reinterpret_cast<double *>(static_cast<char *>(c->ev_d) + 16 +
                                                    (size_t)c->ev_cap * sizeof(int4))
                       : nullptr;
    p.ev_cap = c->ev_cap;
    // the change list after the event list: twice its capacity
    p.chg_len = c->ev_d ? static_cast<int *>(c->ev_d) + 1 : nullptr;
    p.chg = c->ev_d ? reinterpret_cast<int2 *>(static_cast<char *>(c->ev_d) + 16 +
                                               (size_t)c->ev_cap * (sizeof(int4) + 6 * sizeof(double)))
                    : nullptr;
    p.chg_cap = 2 * c->ev_cap;
    p.omega_f = (float)(1.0 / g.tau);
    p.body_xf = (float)g.body_force[0];
    p.body_yf = (float)g.body_force[1];
    p.rho0_f = (float)g.rho0;
    p.wall_ux0_f = (float)g.wall_ux[0];
    p.wall_ux1_f = (float)g.wall_ux[1];
    p.umax_f = (float)g.inflow_umax;
    p.bar = c->bar_d;
    p.spin_limit = c->spin_limit;
    p.near_id = c->near_d;
    return p;
}

void drop_graph(lbm_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
}

void release(lbm_ctx *c) {
    if (!c) return;
    drop_graph(c);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    void *bufs[] = {c->f[0], c->f[1], c->owner, c->flags, c->solids, c->moving_d, c->ring,
                    c->t_d, c->status_d, c->bar_d, c->scratch, c->bnd_d, c->ev_d, c->near_d};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->join) cudaEventDestroy(c->join);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

lbm_status ensure_scratch(lbm_ctx *c, size_t bytes) {
    if (c->scratch_bytes >= bytes) return LBM_OK;
    if (c->scratch) CK(c, cudaFree(c->scratch));
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    CK(c, cudaMalloc(&c->scratch, bytes));
    c->scratch_bytes = bytes;
    return LBM_OK;
}

bool translates(const DSolid &s) { return s.motion == LBM_FREE || s.vx != 0.0 || s.vy != 0.0; }

// Split centres of a solid at rest between steps (R(t) = R(t+1)): at t, at
// t+1, the copy kept through the re-rasterisation and the pair test's
// reference.
void split_centres(DSolid &s) {
    gbm::split_coord(s.x, s.ix0, s.fx0);
    gbm::split_coord(s.y, s.iy0, s.fy0);
    s.ix1 = s.ixo = s.ixt = s.ix0;
    s.iy1 = s.iyo = s.iyt = s.iy0;
    s.fx1 = s.fxo = s.fxt = s.fx0;
    s.fy1 = s.fyo = s.fyt = s.fy0;
}

lbm_status upload_moving(lbm_ctx *c) {
    c->moving.clear();
    for (int s = 0; s < c->nsolid; s++)
        if (c->is_moving[s]) c->moving.push_back(s);
    if ((int)c->moving.size() > c->moving_cap) {
        if (c->moving_d) CK(c, cudaFree(c->moving_d));
        c->moving_d = nullptr;
        c->moving_cap = 0;
        int cap = 64;
        while (cap < (int)c->moving.size()) cap *= 2;
        CK(c, cudaMalloc(&c->moving_d, cap * sizeof(int)));
        c->moving_cap = cap;
    }
    if (!c->moving.empty())
        CK(c, cudaMemcpyAsync(c->moving_d, c->moving.data(), c->moving.size() * sizeof(int),
                              cudaMemcpyHostToDevice, c->stream));
    // event list of the per-solid kernels: SOLID_EVENTS per moving solid (and
    // the change list, twice as long)
    const long long need = (long long)c->moving.size() * gbm::SOLID_EVENTS;
    if (need > c->ev_cap) {
        long long cap = c->ev_cap ? c->ev_cap : 64LL * gbm::SOLID_EVENTS;
        while (cap < need) cap *= 2;
        if (cap > (1LL << 28)) return fail(c, LBM_EINVAL, "too many moving solids");
        CK(c, cudaStreamSynchronize(c->stream));
        if (c->ev_d) CK(c, cudaFree(c->ev_d));
        c->ev_d = nullptr;
        c->ev_cap = 0;
        CK(c, cudaMalloc(&c->ev_d, 16 + (size_t)cap * (sizeof(int4) + 6 * sizeof(double) +
                                                     2 * sizeof(int2))));
        CK(c, cudaMemsetAsync(c->ev_d, 0, 16, c->stream));
        c->ev_cap = (int)cap;
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

// One step t -> t+1: the force kernel (force record of time t, motion) and
// the ring kernel (the moving solids' owner changes and covered/fresh nodes,
// listed) on the side stream beside the advection-collision kernel, all after
// the previous step; then the re-rasterisation of the moving solids (the
// changes applied, refill), which advances t (or a clock tick when no solid
// moves).
lbm_status enqueue_step(lbm_ctx *c, const StepParams &p, bool timed) {
    const bool fork = p.nsolid > 0 && c->overlap;
    if (fork) {
        CK(c, cudaEventRecord(c->fork, c->stream));
        CK(c, cudaStreamWaitEvent(c->side, c->fork, 0));
        CK(c, gbm::launch_forces(p, c->side));
        CK(c, gbm::launch_ring(p, c->side));
        CK(c, cudaEventRecord(c->join, c->side));
        c->launches += p.nmoving > 0 ? 2 : 1;
    } else if (p.nsolid > 0) {
        CK(c, gbm::launch_forces(p, c->stream));
        CK(c, gbm::launch_ring(p, c->stream));
        c->launches += p.nmoving > 0 ? 2 : 1;
    }
    if (timed) {
        if (c->ev_used + 2 > c->ev.size()) {
            for (int k = 0; k < 2; k++) {
                cudaEvent_t e;
                CK(c, cudaEventCreate(&e));
                c->ev.push_back(e);
            }
        }
        CK(c, cudaEventRecord(c->ev[c->ev_used], c->stream));
    }
    CK(c, gbm::launch_stream_collide(p, c->stream));
    if (p.list_by_forces) {  // the slow nodes' update, once the force kernel has listed them
        if (fork) CK(c, cudaStreamWaitEvent(c->stream, c->join, 0));
        CK(c, gbm::launch_deferred_update(p, c->stream));
    }
    if (timed) {
        CK(c, cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
        c->ev_used += 2;
    }
    if (p.L.bc_x == LBM_OPEN) {
        CK(c, gbm::launch_open_columns(p, c->stream));
        c->launches++;
    }
    if (fork && !p.list_by_forces) CK(c, cudaStreamWaitEvent(c->stream, c->join, 0));
    if (p.nmoving > 0) CK(c, gbm::launch_remask(p, c->stream));
    else CK(c, gbm::launch_tick(p, c->stream));
    c->launches += gbm::stream_collide_launches(p) + 1;
    return LBM_OK;
}

lbm_status harvest_timing(lbm_ctx *c) {
    if (c->ev_used == 0) return LBM_OK;
    CK(c, cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
        float ms = 0.f;
        CK(c, cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
        c->timed_ms += ms;
        c->timed_launches++;
    }
    c->ev_used = 0;
    return LBM_OK;
}

lbm_status check_status(lbm_ctx *c) {
    int st = 0;
    CK(c, cudaMemcpyAsync(&st, c->status_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    // a grid barrier that gave up leaves its arrival count behind: clear it
    // whatever else was raised, so that a restored state steps cleanly
    if (st & 4) CK(c, cudaMemsetAsync(c->bar_d, 0, 2 * sizeof(unsigned int), c->stream));
    if (st & 1) return fail(c, LBM_EUNSTABLE, "non-finite or non-positive density produced");
    if (st & 2) return fail(c, LBM_EUNSTABLE, "a solid reached a non-finite state");
    if (st & 4)
        return fail(c, LBM_ETIMEOUT, "a grid-wide barrier of the re-rasterisation kernel gave up");
    if (st & 8)
        return fail(c, LBM_ESTATE,
                    "a solid covered or uncovered more nodes in one step than its event queue "
                    "holds (%d), or the step's owner changes overflowed their list",
                    gbm::SOLID_EVENTS);
    if (st & 16) return fail(c, LBM_ESTATE, "the list of nodes next to solids overflowed");
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_config_default(lbm_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->nx = 64;
    cfg->ny = 64;
    cfg->bc_x = LBM_PERIODIC;
    cfg->bc_y = LBM_PERIODIC;
    cfg->tau = 0.8;
    cfg->rho0 = 1.0;
    cfg->precision = LBM_FP32_DEV;
    cfg->rho_w_mode = LBM_RHOW_CONST;
    cfg->refill = LBM_REFILL_A1;
    cfg->force_ring = 256;
}

lbm_status lbm_create(const lbm_config *cfg, lbm_ctx **out) {
    if (!cfg || !out) return fail(nullptr, LBM_EINVAL, "null argument");
    *out = nullptr;
    const lbm_config &g = *cfg;
    if (g.nx < 4 || g.ny < 4 || (long long)g.nx * g.ny >= (1ll << 31))
        return fail(nullptr, LBM_EINVAL, "domain %d x %d out of range", g.nx, g.ny);
    if (!(g.tau > 0.5) || !std::isfinite(g.tau))
        return fail(nullptr, LBM_EINVAL, "tau must exceed 1/2");
    if (!(g.rho0 > 0.0)) return fail(nullptr, LBM_EINVAL, "rho0 must be positive");
    if (g.bc_x < LBM_PERIODIC || g.bc_x > LBM_OPEN || g.bc_y < LBM_PERIODIC || g.bc_y > LBM_WALL)
        return fail(nullptr, LBM_EINVAL, "invalid boundary kinds");
    if (g.precision < LBM_FP64 || g.precision > LBM_FP16_DEV)
        return fail(nullptr, LBM_EINVAL, "invalid precision");
    if (g.rho_w_mode != LBM_RHOW_CONST && g.rho_w_mode != LBM_RHOW_LOCAL)
        return fail(nullptr, LBM_EINVAL, "invalid rho_w_mode");
    if (g.refill < LBM_REFILL_A1 || g.refill > LBM_REFILL_A3)
        return fail(nullptr, LBM_EINVAL, "invalid refill");
    if (g.force_ring < 1) return fail(nullptr, LBM_EINVAL, "force_ring must be >= 1");
    if (9ll * g.ny * ((g.nx + 63) / 64 * 64) >= (1ll << 31))
        return fail(nullptr, LBM_EINVAL, "domain too large: 9 * ny * pitch must stay below 2^31");
    if (g.motion_cme != 0 && g.motion_cme != 1)
        return fail(nullptr, LBM_EINVAL, "motion_cme must be 0 or 1");
    if (g.relative_changes != 0 && g.relative_changes != 1)
        return fail(nullptr, LBM_EINVAL, "relative_changes must be 0 or 1");
    if (g.collision != LBM_BGK && g.collision != LBM_MRT)
        return fail(nullptr, LBM_EINVAL, "collision must be LBM_BGK or LBM_MRT");
    if (g.collision == LBM_MRT && (g.body_force[0] != 0.0 || g.body_force[1] != 0.0))
        return fail(nullptr, LBM_EINVAL, "MRT takes no body force");
    if (g.boundary != LBM_HALFWAY && g.boundary != LBM_INTERPOLATED)
        return fail(nullptr, LBM_EINVAL, "boundary must be LBM_HALFWAY or LBM_INTERPOLATED");
    if (g.bc_x == LBM_OPEN && g.bc_y != LBM_WALL)
        return fail(nullptr, LBM_EINVAL, "an open channel needs walls in y");
    if (cudaSetDevice(g.device) != cudaSuccess)
        return fail(nullptr, LBM_ECUDA, "cannot select device %d", g.device);

    lbm_ctx *c = new (std::nothrow) lbm_ctx;
    if (!c) return fail(nullptr, LBM_ENOMEM, "host allocation failed");
    c->cfg = g;
    if (g.stream) {
        c->stream = static_cast<cudaStream_t>(g.stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            release(c);
            return fail(nullptr, LBM_ECUDA, "stream creation failed");
        }
        c->own_stream = true;
    }
    c->pitch = (g.nx + 63) / 64 * 64;
    c->elem = elem_bytes(g.precision);
    const size_t plane = (size_t)g.ny * c->pitch;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; b++) e = cudaMalloc(&c->f[b], 9 * plane * c->elem);
    for (int b = 0; b < 2 && e == cudaSuccess; b++)  // row padding stays zero
        e = cudaMemsetAsync(c->f[b], 0, 9 * plane * c->elem, c->stream);
    if (e == cudaSuccess) e = cudaMalloc(&c->owner, plane * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->flags, plane * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->t_d, sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&c->status_d, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->bar_d, 4 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->bar_d, 0, 4 * sizeof(unsigned int), c->stream);
    if (e == cudaSuccess) {
        int lo = 0, hi = 0;  // the force kernel's stream at the highest priority
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->owner, 0xFF, plane * sizeof(uint16_t), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->t_d, 0, sizeof(long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status_d, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) {
        StepParams p = params(c);
        e = gbm::launch_init_populations(p, c->stream);
        if (e == cudaSuccess) e = gbm::launch_flags_all(p, c->stream);
        c->launches += 2;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        lbm_status st = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
        fail(nullptr, st, "lbm_create: %s", cudaGetErrorString(e));
        release(c);
        return st;
    }
    *out = c;
    return LBM_OK;
}

lbm_status lbm_destroy(lbm_ctx *ctx) {
    if (!ctx) return LBM_OK;
    if (ctx->batch) return fail(ctx, LBM_EINVAL, "a case of a batch is destroyed with its batch");
    cudaSetDevice(ctx->cfg.device);
    cudaStreamSynchronize(ctx->stream);
    release(ctx);
    return LBM_OK;
}

lbm_status lbm_add_solid(lbm_ctx *c, const lbm_disk *d, int32_t *id_out) {
    if (!c || !d) return LBM_EINVAL;
    if (c->batch) return fail(c, LBM_EINVAL, "add solids to a batch case with lbm_batch_add_solid");
    const lbm_config &g = c->cfg;
    const double rmax = 0.5 * (g.nx < g.ny ? g.nx : g.ny) - 4.0;
    if (!(d->r > 0.0) || !(d->r < rmax))
        return fail(c, LBM_EINVAL, "radius %g outside (0, %g)", d->r, rmax);
    if (!std::isfinite(d->cx) || !std::isfinite(d->cy) || !std::isfinite(d->vx) ||
        !std::isfinite(d->vy) || !std::isfinite(d->omega))
        return fail(c, LBM_EINVAL, "non-finite disk state");
    if (std::fabs(d->cx) > 1e9 || std::fabs(d->cy) > 1e9)
        return fail(c, LBM_EINVAL, "disk centre too far from the domain");
    if (d->motion != LBM_PRESCRIBED && d->motion != LBM_FREE)
        return fail(c, LBM_EINVAL, "invalid motion");
    if (d->motion == LBM_FREE && !(d->rho_s > 0.0))
        return fail(c, LBM_EINVAL, "a free disk needs rho_s > 0");
    if (d->reserved != 0) return fail(c, LBM_EINVAL, "reserved must be 0");
    if (c->nsolid >= 65534) return fail(c, LBM_EINVAL, "too many solids");
    CK(c, cudaSetDevice(g.device));
    drop_graph(c);
    lbm_status hs = harvest_timing(c);
    if (hs != LBM_OK) return hs;
    if (c->nsolid == c->solid_cap) {
        int cap = c->solid_cap ? 2 * c->solid_cap : 64;
        DSolid *ns = nullptr;
        CK(c, cudaMalloc(&ns, cap * sizeof(DSolid)));
        if (c->nsolid)
            CK(c, cudaMemcpyAsync(ns, c->solids, c->nsolid * sizeof(DSolid),
                                  cudaMemcpyDeviceToDevice, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        if (c->solids) CK(c, cudaFree(c->solids));
        c->solids = ns;
        if (c->near_d) CK(c, cudaFree(c->near_d));  // rebuilt by the next pair test
        c->near_d = nullptr;
        CK(c, cudaMalloc(&c->near_d, (size_t)cap * gbm::NEAR_CAP * sizeof(uint16_t)));
        c->solid_cap = cap;
    }
    if (c->nsolid + 1 > c->ring_cap) {
        int cap = c->ring_cap ? c->ring_cap : 64;
        while (cap < c->nsolid + 1) cap *= 2;
        CK(c, cudaStreamSynchronize(c->stream));
        if (c->ring) CK(c, cudaFree(c->ring));
        c->ring = nullptr;
        c->ring_cap = 0;
        CK(c, cudaMalloc(&c->ring, (size_t)(g.force_ring + 1) * 2 * cap * 3 * sizeof(double)));
        c->ring_cap = cap;
    }
    DSolid s{};
    s.xa = s.x = s.xn = d->cx;
    s.ya = s.y = s.yn = d->cy;
    s.xw = s.xnw = g.bc_x == LBM_PERIODIC ? d->cx - g.nx * std::floor(d->cx / g.nx) : d->cx;
    s.yw = s.ynw = g.bc_y == LBM_PERIODIC ? d->cy - g.ny * std::floor(d->cy / g.ny) : d->cy;
    s.vx = s.vxn = d->vx;
    s.vy = s.vyn = d->vy;
    s.om = s.omn = d->omega;
    s.r = d->r;
    s.rho_s = d->rho_s;
    s.ta = c->t;
    s.xo = s.x;
    s.yo = s.y;
    split_centres(s);
    s.rc = (int)std::ceil(d->r);
    s.r2f = (float)(d->r * d->r);
    s.rmf = 1e-5f * s.r2f + 1e-5f;
    s.ev_t = -1;
    s.near_n = -1;  // until the next pair test: every solid is a neighbour
    s.vxf = (float)d->vx;
    s.vyf = (float)d->vy;
    s.omf = (float)d->omega;
    s.xf = s.xnf = (float)d->cx;
    s.yf = s.ynf = (float)d->cy;
    s.xwi = (int)std::floor(s.xw);
    s.ywi = (int)std::floor(s.yw);
    s.xwr = (float)(s.xw - std::floor(s.xw));
    s.ywr = (float)(s.yw - std::floor(s.yw));
    s.motion = d->motion;
    const int id = c->nsolid;
    CK(c, cudaMemcpyAsync(c->solids + id, &s, sizeof s, cudaMemcpyHostToDevice, c->stream));
    c->nsolid++;
    c->is_moving.push_back(translates(s) ? 1 : 0);
    lbm_status st = upload_moving(c);
    if (st != LBM_OK) return st;
    // room in the deferred per-node list for the new disk's box
    const long long h = gbm::boundary_half(d->r);
    c->bnd_need += (2 * h + 1) * (2 * h + 1);
    if (c->bnd_need > c->bnd_cap) {
        if (c->bnd_need > (1LL << 30)) return fail(c, LBM_EINVAL, "solids too large for the node list");
        long long cap = c->bnd_cap ? c->bnd_cap : 4096;
        while (cap < c->bnd_need) cap *= 2;
        CK(c, cudaStreamSynchronize(c->stream));
        if (c->bnd_d) CK(c, cudaFree(c->bnd_d));
        c->bnd_d = nullptr;
        c->bnd_cap = 0;
        CK(c, cudaMalloc(&c->bnd_d, (size_t)(cap + 2) * sizeof(int)));
        CK(c, cudaMemsetAsync(c->bnd_d, 0, 2 * sizeof(int), c->stream));
        c->bnd_cap = (int)cap;
    }
    CK(c, cudaMemsetAsync(c->bar_d + 3, 1, sizeof(unsigned int), c->stream));  // pair test
    StepParams p = params(c);
    CK(c, gbm::launch_stamp_solid(p, id, c->stream));
    c->launches += 2;
    CK(c, cudaStreamSynchronize(c->stream));
    c->ring_base = c->t;  // the record layout changed with nsolid
    if (id_out) *id_out = id;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *c, int64_t n) {
    if (!c || n < 0) return LBM_EINVAL;
    if (c->batch) return fail(c, LBM_EINVAL, "a case of a batch is stepped by lbm_batch_run");
    CK(c, cudaSetDevice(c->cfg.device));
    const StepParams p = params(c);
    int64_t done = 0;
    const bool graphs = c->graph_steps > 1 && !c->timing;
    if (graphs) {
        while (n - done >= c->graph_steps) {
            if (!c->gexec) {
                cudaGraph_t graph;
                CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
                const int64_t before = c->launches;
                for (int k = 0; k < c->graph_steps; k++) {
                    lbm_status st = enqueue_step(c, p, false);
                    if (st != LBM_OK) {
                        cudaStreamEndCapture(c->stream, &graph);
                        return st;
                    }
                }
                c->graph_launches = c->launches - before;
                c->launches = before;  // counted when the graph is launched
                CK(c, cudaStreamEndCapture(c->stream, &graph));
                cudaError_t e = cudaGraphInstantiate(&c->gexec, graph, 0);
                cudaGraphDestroy(graph);
                CK(c, e);
            }
            CK(c, cudaGraphLaunch(c->gexec, c->stream));
            c->launches += c->graph_launches;
            done += c->graph_steps;
        }
    }
    for (; done < n; done++) {
        lbm_status st = enqueue_step(c, p, c->timing);
        if (st != LBM_OK) return st;
        if (c->timing && c->ev_used >= 8192) {
            st = harvest_timing(c);
            if (st != LBM_OK) return st;
        }
    }
    c->t += n;
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx *c) {
    if (!c) return LBM_EINVAL;
    CK(c, cudaSetDevice(c->cfg.device));
    CK(c, cudaStreamSynchronize(c->stream));
    return check_status(c);
}

lbm_status lbm_forces(lbm_ctx *c, int32_t form, int64_t first, int64_t count, double *out,
                      int32_t on_device) {
    if (!c || (form != LBM_CME && form != LBM_GME) || count < 0 || (!out && count > 0))
        return LBM_EINVAL;
    const int64_t lo = c->t - c->cfg.force_ring > c->ring_base ? c->t - c->cfg.force_ring
                                                                : c->ring_base;
    if (first < lo || first + count > c->t)
        return fail(c, LBM_ESTATE, "records %lld..%lld not available (have %lld..%lld)",
                    (long long)first, (long long)(first + count - 1), (long long)lo,
                    (long long)(c->t - 1));
    CK(c, cudaSetDevice(c->cfg.device));
    const int ns = c->nsolid;
    if (ns > 0 && count > 0) {
        const size_t w = (size_t)ns * 3 * sizeof(double);
        int64_t k = 0;
        const int64_t slots = c->cfg.force_ring + 1;
        while (k < count) {
            const int64_t slot = (first + k) % slots;
            int64_t run = slots - slot;
            if (run > count - k) run = count - k;
            const double *src = c->ring + ((size_t)slot * 2 + form) * ns * 3;
            CK(c, cudaMemcpy2DAsync(out + (size_t)k * ns * 3, w, src, 2 * w, w, (size_t)run,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    c->stream));
            k += run;
        }
    }
    if (!on_device) return lbm_sync(c);
    return LBM_OK;
}

lbm_status lbm_fields(lbm_ctx *c, double *rho, double *ux, double *uy, int32_t on_device) {
    if (!c || !rho || !ux || !uy) return LBM_EINVAL;
    CK(c, cudaSetDevice(c->cfg.device));
    const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
    const StepParams p = params(c);
    if (on_device) {
        CK(c, gbm::launch_fields(p, rho, ux, uy, c->stream));
        c->launches++;
        return LBM_OK;
    }
    lbm_status st = ensure_scratch(c, 3 * n * sizeof(double));
    if (st != LBM_OK) return st;
    double *s = static_cast<double *>(c->scratch);
    CK(c, gbm::launch_fields(p, s, s + n, s + 2 * n, c->stream));
    c->launches++;
    CK(c, cudaMemcpyAsync(rho, s, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(ux, s + n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(uy, s + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return lbm_sync(c);
}

}  // extern "C"

// Fixed staging array of lbm_fields_static: rho, ux, uy of up to
// LBM_FIELDS_STATIC_MAX_NODES nodes, reserved on every device that loads the
// library.  Host code must not use the symbol itself as a device address; the
// address is looked up once per device below.
static __device__ __align__(256) double g_fields_stage[3 * LBM_FIELDS_STATIC_MAX_NODES];

namespace {
constexpr int MAX_DEVICES = 64;
std::mutex g_stage_mutex;
double *g_stage_ptr[MAX_DEVICES] = {};
}  // namespace

extern "C" {

lbm_status lbm_fields_static(lbm_ctx *c, double *rho, double *ux, double *uy) {
    if (!c || !rho || !ux || !uy) return LBM_EINVAL;
    const int dev = c->cfg.device;
    const long long n = (long long)c->cfg.nx * c->cfg.ny;
    if (n > LBM_FIELDS_STATIC_MAX_NODES)
        return fail(c, LBM_EINVAL, "lbm_fields_static: %lld nodes exceed the fixed maximum of %d",
                    n, LBM_FIELDS_STATIC_MAX_NODES);
    if (dev < 0 || dev >= MAX_DEVICES) return fail(c, LBM_EINVAL, "device ordinal out of range");
    CK(c, cudaSetDevice(dev));
    double *stage = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_stage_mutex);
        if (!g_stage_ptr[dev]) {
            void *ptr = nullptr;
            CK(c, cudaGetSymbolAddress(&ptr, g_fields_stage));
            g_stage_ptr[dev] = static_cast<double *>(ptr);
        }
        stage = g_stage_ptr[dev];
    }
    const StepParams p = params(c);
    CK(c, gbm::launch_fields(p, stage, stage + n, stage + 2 * n, c->stream));
    c->launches++;
    CK(c, cudaMemcpyAsync(rho, stage, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(ux, stage + n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(uy, stage + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost,
                          c->stream));
    return lbm_sync(c);
}

}  // extern "C"

// ---------------------------------------------------------- checkpoints

namespace {

constexpr uint32_t STATE_MAGIC = 0x534D424Cu;  // "LBMS"
constexpr uint32_t STATE_VERSION = 1;

// Leading block of a saved state; the arrays follow in the order of
// state_parts.  The configuration is kept with its stream and device cleared.
struct StateHeader {
    uint32_t magic, version;
    uint32_t solid_bytes, reserved;
    lbm_config cfg;
    int64_t t, ring_base;
    int32_t pitch, nsolid, ev_len, pad;
};

struct Part {
    char *host;        // position in the caller's buffer
    void *dev;         // device array
    size_t bytes;
};

lbm_config comparable(lbm_config g) {
    g.stream = nullptr;
    g.device = 0;
    return g;
}

int64_t state_bytes(const lbm_ctx *c, int ev_len) {
    const size_t plane = (size_t)c->cfg.ny * c->pitch;
    return (int64_t)(sizeof(StateHeader) + 9 * plane * c->elem + 2 * plane * sizeof(uint16_t) +
                     (size_t)c->nsolid * sizeof(DSolid) +
                     (size_t)(c->cfg.force_ring + 1) * 2 * c->nsolid * 3 * sizeof(double) +
                     (size_t)ev_len * (sizeof(int4) + 6 * sizeof(double)) + (size_t)c->nsolid);
}

// The device arrays of a state, laid out after the header at base.
std::vector<Part> state_parts(lbm_ctx *c, char *base, int ev_len) {
    const size_t plane = (size_t)c->cfg.ny * c->pitch;
    const StepParams p = params(c);
    char *at = base + sizeof(StateHeader);
    std::vector<Part> v;
    auto add = [&](void *dev, size_t bytes) {
        v.push_back(Part{at, dev, bytes});
        at += bytes;
    };
    add((c->t & 1) ? c->f[1] : c->f[0], 9 * plane * c->elem);  // populations of time t
    add(c->owner, plane * sizeof(uint16_t));
    add(c->flags, plane * sizeof(uint16_t));
    add(c->solids, (size_t)c->nsolid * sizeof(DSolid));
    add(c->ring, (size_t)(c->cfg.force_ring + 1) * 2 * c->nsolid * 3 * sizeof(double));
    add(p.ev, (size_t)ev_len * sizeof(int4));
    add(p.ev_mom, (size_t)ev_len * 6 * sizeof(double));
    return v;
}

lbm_status event_count(lbm_ctx *c, int *n) {
    *n = 0;
    if (c->ev_d) {
        CK(c, cudaMemcpyAsync(n, c->ev_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        if (*n > c->ev_cap) *n = c->ev_cap;
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_state_size(lbm_ctx *c, int64_t *bytes) {
    if (!c || !bytes) return LBM_EINVAL;
    CK(c, cudaSetDevice(c->cfg.device));
    int n = 0;
    lbm_status st = event_count(c, &n);
    if (st != LBM_OK) return st;
    *bytes = state_bytes(c, n);
    return LBM_OK;
}

lbm_status lbm_save(lbm_ctx *c, void *buf, int64_t bytes) {
    if (!c || !buf) return LBM_EINVAL;
    if (c->batch) return fail(c, LBM_EINVAL, "a case of a batch is saved with its batch");
    CK(c, cudaSetDevice(c->cfg.device));
    lbm_status st = lbm_sync(c);  // a state with a raised status is not worth keeping
    if (st != LBM_OK) return st;
    int n = 0;
    st = event_count(c, &n);
    if (st != LBM_OK) return st;
    if (bytes < state_bytes(c, n))
        return fail(c, LBM_EINVAL, "buffer of %lld bytes, the state needs %lld", (long long)bytes,
                    (long long)state_bytes(c, n));
    char *base = static_cast<char *>(buf);
    StateHeader h{};
    h.magic = STATE_MAGIC;
    h.version = STATE_VERSION;
    h.solid_bytes = sizeof(DSolid);
    h.cfg = comparable(c->cfg);
    h.t = c->t;
    h.ring_base = c->ring_base;
    h.pitch = c->pitch;
    h.nsolid = c->nsolid;
    h.ev_len = n;
    std::memcpy(base, &h, sizeof h);
    std::vector<Part> parts = state_parts(c, base, n);
    for (const Part &q : parts)
        if (q.bytes) CK(c, cudaMemcpyAsync(q.host, q.dev, q.bytes, cudaMemcpyDeviceToHost, c->stream));
    char *mv = parts.back().host + parts.back().bytes;
    for (int s = 0; s < c->nsolid; s++) mv[s] = (char)c->is_moving[s];
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_load(lbm_ctx *c, const void *buf, int64_t bytes) {
    if (!c || !buf || bytes < (int64_t)sizeof(StateHeader)) return LBM_EINVAL;
    if (c->batch) return fail(c, LBM_EINVAL, "a case of a batch is loaded with its batch");
    StateHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (h.magic != STATE_MAGIC || h.version != STATE_VERSION || h.solid_bytes != sizeof(DSolid))
        return fail(c, LBM_EINVAL, "not a state saved by this library");
    const lbm_config want = comparable(c->cfg);
    if (std::memcmp(&h.cfg, &want, sizeof want) != 0 || h.pitch != c->pitch)
        return fail(c, LBM_EINVAL, "the state was saved with another configuration");
    if (h.nsolid != c->nsolid)
        return fail(c, LBM_EINVAL, "the state has %d solids, the context %d", h.nsolid, c->nsolid);
    if (h.ev_len < 0 || bytes < state_bytes(c, h.ev_len))
        return fail(c, LBM_EINVAL, "truncated state");
    CK(c, cudaSetDevice(c->cfg.device));
    CK(c, cudaStreamSynchronize(c->stream));
    drop_graph(c);
    lbm_status st = harvest_timing(c);
    if (st != LBM_OK) return st;
    const char *base = static_cast<const char *>(buf);
    const char *mv = base + state_bytes(c, h.ev_len) - c->nsolid;
    for (int s = 0; s < c->nsolid; s++) c->is_moving[s] = mv[s] ? 1 : 0;
    st = upload_moving(c);  // also sizes the event list
    if (st != LBM_OK) return st;
    if (h.ev_len > c->ev_cap) return fail(c, LBM_EINVAL, "the state's event list does not fit");
    c->t = h.t;
    c->ring_base = h.ring_base;
    std::vector<Part> parts = state_parts(c, const_cast<char *>(base), h.ev_len);
    for (const Part &q : parts)
        if (q.bytes) CK(c, cudaMemcpyAsync(q.dev, q.host, q.bytes, cudaMemcpyHostToDevice, c->stream));
    const long long t = h.t;
    CK(c, cudaMemcpyAsync(c->t_d, &t, sizeof t, cudaMemcpyHostToDevice, c->stream));
    if (c->ev_d) CK(c, cudaMemcpyAsync(c->ev_d, &h.ev_len, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    // clean control words: status, barrier, displacement; a pair test first
    const unsigned int ctl[4] = {0u, 0u, 0u, 1u};
    CK(c, cudaMemcpyAsync(c->bar_d, ctl, sizeof ctl, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemsetAsync(c->status_d, 0, sizeof(int), c->stream));
    if (c->bnd_d) CK(c, cudaMemsetAsync(c->bnd_d, 0, 2 * sizeof(int), c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

}  // extern "C"

extern "C" {

lbm_status lbm_get_populations(lbm_ctx *c, double *f, int32_t on_device) {
    if (!c || !f) return LBM_EINVAL;
    CK(c, cudaSetDevice(c->cfg.device));
    const size_t n = 9 * (size_t)c->cfg.nx * c->cfg.ny;
    const StepParams p = params(c);
    if (on_device) {
        CK(c, gbm::launch_export_populations(p, f, c->stream));
        c->launches++;
        return LBM_OK;
    }
    lbm_status st = ensure_scratch(c, n * sizeof(double));
    if (st != LBM_OK) return st;
    CK(c, gbm::launch_export_populations(p, static_cast<double *>(c->scratch), c->stream));
    c->launches++;
    CK(c, cudaMemcpyAsync(f, c->scratch, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return lbm_sync(c);
}

lbm_status lbm_set_populations(lbm_ctx *c, const double *f, int32_t on_device) {
    if (!c || !f) return LBM_EINVAL;
    CK(c, cudaSetDevice(c->cfg.device));
    const size_t n = 9 * (size_t)c->cfg.nx * c->cfg.ny;
    const StepParams p = params(c);
    if (on_device) {
        CK(c, gbm::launch_import_populations(p, f, c->stream));
        c->launches++;
        return LBM_OK;
    }
    lbm_status st = ensure_scratch(c, n * sizeof(double));
    if (st != LBM_OK) return st;
    CK(c, cudaMemcpyAsync(c->scratch, f, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(c, gbm::launch_import_populations(p, static_cast<const double *>(c->scratch), c->stream));
    c->launches++;
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_warm_start(lbm_ctx *c, const float *pred, double u_scale, double rho_scale,
                          int32_t flags) {
    if (!c || !pred || !std::isfinite(u_scale) || !std::isfinite(rho_scale) || flags < 0 ||
        flags > (LBM_WS_BASE | LBM_WS_FLUX))
        return LBM_EINVAL;
    if (flags && c->cfg.bc_x != LBM_OPEN)
        return fail(c, LBM_EINVAL, "a Poiseuille base needs an open channel");
    if ((flags & LBM_WS_FLUX) && !(flags & LBM_WS_BASE))
        return fail(c, LBM_EINVAL, "the column flux correction works on the Poiseuille base");
    const int base = flags;
    CK(c, cudaSetDevice(c->cfg.device));
    CK(c, gbm::launch_warm_start(params(c), pred, u_scale, rho_scale, base, c->stream));
    c->launches++;
    return LBM_OK;
}

lbm_status lbm_case_input(lbm_ctx *c, double reynolds, float *in) {
    if (!c || !in || !(reynolds > 0.0) || !std::isfinite(reynolds)) return LBM_EINVAL;
    CK(c, cudaSetDevice(c->cfg.device));
    CK(c, gbm::launch_case_features(params(c), reynolds, in, c->stream));
    c->launches++;
    return LBM_OK;
}

lbm_status lbm_get_owner(lbm_ctx *c, int32_t *owner, int32_t on_device) {
    if (!c || !owner) return LBM_EINVAL;
    CK(c, cudaSetDevice(c->cfg.device));
    const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
    const StepParams p = params(c);
    if (on_device) {
        CK(c, gbm::launch_export_owner(p, owner, c->stream));
        c->launches++;
        return LBM_OK;
    }
    lbm_status st = ensure_scratch(c, n * sizeof(int32_t));
    if (st != LBM_OK) return st;
    CK(c, gbm::launch_export_owner(p, static_cast<int32_t *>(c->scratch), c->stream));
    c->launches++;
    CK(c, cudaMemcpyAsync(owner, c->scratch, n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                          c->stream));
    return lbm_sync(c);
}

lbm_status lbm_get_solids(lbm_ctx *c, double *state) {
    if (!c || (!state && c->nsolid > 0)) return LBM_EINVAL;
    if (c->nsolid == 0) return LBM_OK;
    CK(c, cudaSetDevice(c->cfg.device));
    std::vector<DSolid> h(c->nsolid);
    CK(c, cudaMemcpyAsync(h.data(), c->solids, c->nsolid * sizeof(DSolid), cudaMemcpyDeviceToHost,
                          c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    for (int s = 0; s < c->nsolid; s++) {
        double *o = state + 5 * s;
        o[0] = h[s].x;
        o[1] = h[s].y;
        o[2] = h[s].vx;
        o[3] = h[s].vy;
        o[4] = h[s].om;
    }
    return LBM_OK;
}

lbm_status lbm_set_solid(lbm_ctx *c, int32_t id, const double *state) {
    if (!c || !state || id < 0 || id >= c->nsolid) return LBM_EINVAL;
    if (c->batch) return fail(c, LBM_EINVAL, "solids of a batch case rest");
    for (int k = 0; k < 5; k++)
        if (!std::isfinite(state[k])) return fail(c, LBM_EINVAL, "non-finite solid state");
    CK(c, cudaSetDevice(c->cfg.device));
    DSolid s;
    CK(c, cudaMemcpyAsync(&s, c->solids + id, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (state[0] != s.x || state[1] != s.y)
        return fail(c, LBM_EINVAL, "lbm_set_solid changes velocities only; position must match");
    s.xa = s.xn = s.xo = s.x;
    s.ya = s.yn = s.yo = s.y;
    split_centres(s);
    s.ta = c->t;
    s.vx = s.vxn = state[2];
    s.vy = s.vyn = state[3];
    s.om = s.omn = state[4];
    s.vxf = (float)state[2];
    s.vyf = (float)state[3];
    s.omf = (float)state[4];
    CK(c, cudaMemcpyAsync(c->solids + id, &s, sizeof s, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemsetAsync(c->bar_d + 3, 1, sizeof(unsigned int), c->stream));  // pair test
    drop_graph(c);
    c->is_moving[id] = translates(s) ? 1 : 0;
    return upload_moving(c);
}

lbm_status lbm_links(lbm_ctx *c, int64_t cap, int32_t *out, int64_t *n_out) {
    if (!c || cap < 0 || (!out && cap > 0)) return LBM_EINVAL;
    CK(c, cudaSetDevice(c->cfg.device));
    const int nx = c->cfg.nx, ny = c->cfg.ny;
    const size_t n = (size_t)nx * ny;
    lbm_status st = ensure_scratch(c, n * (sizeof(int32_t) + 1));
    if (st != LBM_OK) return st;
    const StepParams p = params(c);
    int32_t *own_d = static_cast<int32_t *>(c->scratch);
    uint8_t *mask_d = reinterpret_cast<uint8_t *>(own_d + n);
    CK(c, gbm::launch_export_owner(p, own_d, c->stream));
    CK(c, gbm::launch_link_masks(p, mask_d, c->stream));
    c->launches += 2;
    std::vector<int32_t> own(n);
    std::vector<uint8_t> mask(n);
    CK(c, cudaMemcpyAsync(own.data(), own_d, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(mask.data(), mask_d, n, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    static const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    static const int ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    int64_t k = 0;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            const uint8_t m = mask[(size_t)y * nx + x];
            if (!m) continue;
            for (int i = 1; i < 9; i++) {
                if (!((m >> (i - 1)) & 1)) continue;
                if (k < cap) {
                    const int xb = (x + ex[i] + nx) % nx, yb = (y + ey[i] + ny) % ny;
                    out[4 * k] = x;
                    out[4 * k + 1] = y;
                    out[4 * k + 2] = i;
                    out[4 * k + 3] = own[(size_t)yb * nx + xb];
                }
                k++;
            }
        }
    if (n_out) *n_out = k;
    return LBM_OK;
}

int64_t lbm_time(const lbm_ctx *c) { return c ? c->t : -1; }
int32_t lbm_nsolid(const lbm_ctx *c) { return c ? c->nsolid : -1; }

const char *lbm_last_error(const lbm_ctx *c) {
    return c ? c->err.c_str() : g_create_error.c_str();
}

const char *lbm_status_string(lbm_status st) {
    switch (st) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument";
        case LBM_ENOMEM: return "out of memory";
        case LBM_ECUDA: return "CUDA error";
        case LBM_EUNSTABLE: return "unstable (non-finite density)";
        case LBM_ETIMEOUT: return "device wait timed out";
        case LBM_ESTATE: return "invalid state";
    }
    return "unknown status";
}

lbm_status lbm_set_wait_limit(lbm_ctx *c, int64_t polls) {
    if (!c || polls < 0) return LBM_EINVAL;
    if (c->batch) return fail(c, LBM_EINVAL, "a case of a batch is stepped by its batch");
    c->spin_limit = polls;
    drop_graph(c);  // captured launches carry the old limit
    return LBM_OK;
}

lbm_status lbm_set_graph(lbm_ctx *c, int32_t steps_per_graph) {
    if (!c || steps_per_graph < 0) return LBM_EINVAL;
    if (steps_per_graph > 1 && !c->own_stream && c->stream == nullptr)
        return fail(c, LBM_EINVAL, "graphs need a non-default stream");
    drop_graph(c);
    c->graph_steps = steps_per_graph;
    return LBM_OK;
}

lbm_status lbm_set_timing(lbm_ctx *c, int32_t enable) {
    if (!c) return LBM_EINVAL;
    lbm_status st = harvest_timing(c);
    if (st != LBM_OK) return st;
    c->timing = enable != 0;
    c->timed_ms = 0.0;
    c->timed_launches = 0;
    return LBM_OK;
}

lbm_status lbm_get_timing(lbm_ctx *c, double *ms, int64_t *launches) {
    if (!c) return LBM_EINVAL;
    lbm_status st = harvest_timing(c);
    if (st != LBM_OK) return st;
    if (ms) *ms = c->timed_ms;
    if (launches) *launches = c->timed_launches;
    return LBM_OK;
}

int64_t lbm_launch_count(const lbm_ctx *c) { return c ? c->launches : -1; }

lbm_status lbm_set_kernel_variant(lbm_ctx *c, int32_t variant) {
    if (!c || variant < 0 || variant >= gbm::KERNEL_VARIANTS) return LBM_EINVAL;
    drop_graph(c);
    c->sc_variant = variant;
    // the deferred list's lengths are kept only while the deferred path runs
    if (c->bnd_d) CK(c, cudaMemsetAsync(c->bnd_d, 0, 2 * sizeof(int), c->stream));
    return LBM_OK;
}

int32_t lbm_kernel_variant(const lbm_ctx *c) { return c ? c->sc_variant : -1; }

lbm_status lbm_set_force_overlap(lbm_ctx *c, int32_t on) {
    if (!c || (on != 0 && on != 1)) return LBM_EINVAL;
    drop_graph(c);
    c->overlap = on != 0;
    return LBM_OK;
}

int32_t lbm_force_overlap(const lbm_ctx *c) { return c ? (c->overlap ? 1 : 0) : -1; }

lbm_status lbm_autotune(lbm_ctx *c, int32_t steps, int32_t *best) {
    if (!c || steps < 1) return LBM_EINVAL;
    if (c->batch) return fail(c, LBM_EINVAL, "a case of a batch is tuned by lbm_batch_autotune");
    CK(c, cudaSetDevice(c->cfg.device));
    const bool was_timing = c->timing;
    const int keep_graph = c->graph_steps;
    lbm_status st = harvest_timing(c);
    if (st != LBM_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(c, cudaEventCreate(&e0));
    CK(c, cudaEventCreate(&e1));
    c->timing = false;
    c->graph_steps = 0;
    double best_ms = 0.0;
    int best_v = 0;
    bool best_o = true;
    for (int o = 1; o >= 0 && st == LBM_OK; o--) {
        for (int v = 0; v < gbm::KERNEL_VARIANTS && st == LBM_OK; v++) {
            c->sc_variant = v;
            c->overlap = o != 0;
            drop_graph(c);
            if (c->bnd_d) CK(c, cudaMemsetAsync(c->bnd_d, 0, 2 * sizeof(int), c->stream));
            st = lbm_step(c, 1);  // the first step of a shape is not timed
            if (st == LBM_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) st = LBM_ECUDA;
            if (st == LBM_OK) st = lbm_step(c, steps);
            if (st == LBM_OK && cudaEventRecord(e1, c->stream) != cudaSuccess) st = LBM_ECUDA;
            if (st == LBM_OK) st = lbm_sync(c);
            float ms = 0.f;
            if (st == LBM_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = LBM_ECUDA;
            if (st == LBM_OK && ((o == 1 && v == 0) || ms < best_ms)) {
                best_ms = ms;
                best_v = v;
                best_o = o != 0;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->sc_variant = best_v;
    c->overlap = best_o;
    drop_graph(c);
    if (c->bnd_d) cudaMemsetAsync(c->bnd_d, 0, 2 * sizeof(int), c->stream);
    c->timing = was_timing;
    c->graph_steps = keep_graph;
    if (st != LBM_OK) return st == LBM_ECUDA ? fail(c, st, "autotuner: event timing failed") : st;
    if (best) *best = best_v;
    return LBM_OK;
}

}  // extern "C"

// ====================================================================== batch
//
// A batch owns ncase ordinary contexts (its cases) that share one stream, and
// steps all of them with three kernels: the fused advection-collision kernel
// over the list of active tiles {case, x block, row}, the force kernel over
// the list of active (case, solid) items (which also advances the step
// counters), and every `every` steps the convergence kernel, which retires
// cases and rebuilds both lists on the device, so that a captured graph of
// `every` steps stays valid while cases retire.

struct lbm_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<lbm_ctx *> cases;
    int precision = 0, rho_w_mode = 0;
    bool force = false;
    // launch policy
    int variant = 0;
    int tile_h = 1;  // rows per tile of the fused kernel
    bool persistent = false, graph = true;
    // convergence test
    int every = 100;
    double tol = 1e-7;
    int64_t max_steps = 2000000;
    int since_test = 0;  // batch steps since the last test
    // device tables
    bool dirty = true;  // parameters or lists must be rebuilt before stepping
    bool uploaded = false;  // cases_d holds parameters (with the f0 = current convention)
    StepParams *cases_d = nullptr;
    int4 *tiles_d = nullptr;
    int2 *items_d = nullptr;
    int *counts_d = nullptr;  // {ntiles, nitems, nactive}
    int *active_d = nullptr;
    unsigned int *ticket_d = nullptr;
    int *state_d = nullptr;
    double *drag_d = nullptr;
    int *calm_d = nullptr;       // tests in a row within tol of the anchor, per case
    double *anchor_d = nullptr;  // drag at the start of that run, per case
    int window = 1;              // tests in a row within tol that retire a case
    long long *steps_d = nullptr;
    int *toff_d = nullptr, *ioff_d = nullptr;
    long long tile_cap = 0, item_cap = 0;
    int max_tiles = 0, max_items = 0;
    int *nactive_h = nullptr;  // pinned
    // host copies of the per-case results
    std::vector<int32_t> state;
    std::vector<long long> steps;
    std::vector<double> drag;
    cudaGraphExec_t gexec = nullptr;
    // timing of the fused kernel
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    double timed_ms = 0.0;
    int64_t timed_launches = 0;
    int64_t launches = 0;
    std::string err;
};

namespace {

lbm_status bfail(lbm_batch *b, lbm_status st, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
lbm_status bfail(lbm_batch *b, lbm_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_create_error = buf;
    return st;
}

#define BCK(b, call)                                                                        \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,     \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                  \
    } while (0)

gbm::BatchLaunch blaunch(const lbm_batch *b) {
    gbm::BatchLaunch l{};
    l.cases = b->cases_d;
    l.tiles = b->tiles_d;
    l.ntiles = b->counts_d;
    l.items = b->items_d;
    l.nitems = b->counts_d + 1;
    l.active = b->active_d;
    l.nactive = b->counts_d + 2;
    l.ticket = b->ticket_d;
    l.precision = b->precision;
    l.variant = b->variant;
    l.force = b->force;
    l.local = b->rho_w_mode == LBM_RHOW_LOCAL;
    l.max_items = b->max_items;
    l.max_tiles = b->max_tiles;
    l.tile_h = b->tile_h;
    l.persistent = b->persistent;
    return l;
}

gbm::BatchState bstate(const lbm_batch *b) {
    gbm::BatchState s{};
    s.ncase = (int)b->cases.size();
    s.tol = b->tol;
    s.max_steps = b->max_steps;
    s.state = b->state_d;
    s.drag = b->drag_d;
    s.window = b->window;
    s.calm = b->calm_d;
    s.anchor = b->anchor_d;
    s.steps = b->steps_d;
    s.toff = b->toff_d;
    s.ioff = b->ioff_d;
    return s;
}

void bdrop_graph(lbm_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
}

void brelease(lbm_batch *b) {
    if (!b) return;
    bdrop_graph(b);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    for (lbm_ctx *c : b->cases) {
        c->batch = nullptr;
        release(c);
    }
    void *bufs[] = {b->cases_d, b->tiles_d, b->items_d, b->counts_d, b->active_d, b->ticket_d,
                    b->state_d, b->drag_d, b->calm_d, b->anchor_d, b->steps_d, b->toff_d,
                    b->ioff_d};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (b->nactive_h) cudaFreeHost(b->nactive_h);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// Upload the case parameters and rebuild the lists (clears the drag history).
lbm_status bprepare(lbm_batch *b) {
    if (!b->dirty) return LBM_OK;
    bdrop_graph(b);
    if (b->uploaded) {
        // the cases' clocks moved on the device: the buffer holding the
        // current populations follows the parity of each clock
        const size_t n = b->cases.size();
        BCK(b, gbm::launch_batch_converge(blaunch(b), bstate(b), gbm::BATCH_GATHER, b->stream));
        b->launches++;
        BCK(b, cudaMemcpyAsync(b->steps.data(), b->steps_d, n * sizeof(long long),
                               cudaMemcpyDeviceToHost, b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
        for (size_t k = 0; k < n; k++) b->cases[k]->t = b->steps[k];
    }
    const int w = gbm::tile_nodes(b->precision, b->variant);
    const int wmin = gbm::tile_nodes(b->precision, 2);
    long long tiles = 0, tiles_min = 0, items = 0;
    std::vector<StepParams> hp(b->cases.size());
    for (size_t k = 0; k < b->cases.size(); k++) {
        const lbm_ctx *c = b->cases[k];
        tiles += (long long)((c->cfg.nx + w - 1) / w) * ((c->cfg.ny + b->tile_h - 1) / b->tile_h);
        tiles_min += (long long)((c->cfg.nx + wmin - 1) / wmin) * c->cfg.ny;
        items += c->nsolid;
        hp[k] = params(c);
        hp[k].sc_variant = b->variant;
        if (c->t & 1) {  // batch convention: f0 holds the current populations
            hp[k].f0 = c->f[1];
            hp[k].f1 = c->f[0];
        }
    }
    if (tiles_min >= (1ll << 31) || items >= (1ll << 31))
        return bfail(b, LBM_EINVAL, "batch too large: %lld tiles", tiles_min);
    BCK(b, cudaStreamSynchronize(b->stream));
    if (tiles_min > b->tile_cap) {
        if (b->tiles_d) BCK(b, cudaFree(b->tiles_d));
        b->tiles_d = nullptr;
        b->tile_cap = 0;
        BCK(b, cudaMalloc(&b->tiles_d, (size_t)tiles_min * sizeof(int4)));
        b->tile_cap = tiles_min;
    }
    if (items > b->item_cap || !b->items_d) {
        if (b->items_d) BCK(b, cudaFree(b->items_d));
        b->items_d = nullptr;
        b->item_cap = 0;
        const long long cap = items > 0 ? items : 1;
        BCK(b, cudaMalloc(&b->items_d, (size_t)cap * sizeof(int2)));
        b->item_cap = cap;
    }
    b->max_tiles = (int)tiles;
    b->max_items = (int)items;
    BCK(b, cudaMemcpyAsync(b->cases_d, hp.data(), hp.size() * sizeof(StepParams),
                           cudaMemcpyHostToDevice, b->stream));
    BCK(b, gbm::launch_batch_converge(blaunch(b), bstate(b), gbm::BATCH_REBUILD, b->stream));
    b->launches++;
    BCK(b, cudaMemcpyAsync(b->nactive_h, b->counts_d + 2, sizeof(int), cudaMemcpyDeviceToHost,
                           b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));  // hp must outlive the copy
    b->since_test = 0;
    b->dirty = false;
    b->uploaded = true;
    return LBM_OK;
}

lbm_status benqueue_step(lbm_batch *b, const gbm::BatchLaunch &l, bool timed) {
    if (timed) {
        if (b->ev_used + 2 > b->ev.size()) {
            for (int k = 0; k < 2; k++) {
                cudaEvent_t e;
                BCK(b, cudaEventCreate(&e));
                b->ev.push_back(e);
            }
        }
        BCK(b, cudaEventRecord(b->ev[b->ev_used], b->stream));
    }
    BCK(b, gbm::launch_stream_collide_batch(l, b->stream));
    if (timed) {
        BCK(b, cudaEventRecord(b->ev[b->ev_used + 1], b->stream));
        b->ev_used += 2;
    }
    BCK(b, gbm::launch_solids_batch(l, b->stream));
    b->launches += 2;
    return LBM_OK;
}

lbm_status bharvest(lbm_batch *b) {
    if (b->ev_used == 0) return LBM_OK;
    BCK(b, cudaStreamSynchronize(b->stream));
    for (size_t k = 0; k + 1 < b->ev_used; k += 2) {
        float ms = 0.f;
        BCK(b, cudaEventElapsedTime(&ms, b->ev[k], b->ev[k + 1]));
        b->timed_ms += ms;
        b->timed_launches++;
    }
    b->ev_used = 0;
    return LBM_OK;
}

// Step counters, states and drags to the host; the cases' clocks follow.
lbm_status bgather(lbm_batch *b) {
    const size_t n = b->cases.size();
    lbm_status st = bprepare(b);  // the kernel reads the uploaded case parameters
    if (st != LBM_OK) return st;
    BCK(b, gbm::launch_batch_converge(blaunch(b), bstate(b), gbm::BATCH_GATHER, b->stream));
    b->launches++;
    BCK(b, cudaMemcpyAsync(b->state.data(), b->state_d, n * sizeof(int), cudaMemcpyDeviceToHost,
                           b->stream));
    BCK(b, cudaMemcpyAsync(b->steps.data(), b->steps_d, n * sizeof(long long),
                           cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaMemcpyAsync(b->drag.data(), b->drag_d, n * sizeof(double), cudaMemcpyDeviceToHost,
                           b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    for (size_t k = 0; k < n; k++) b->cases[k]->t = b->steps[k];
    return LBM_OK;
}

// `n` steps of every active case, without a convergence test.
lbm_status bsteps(lbm_batch *b, int64_t n) {
    const gbm::BatchLaunch l = blaunch(b);
    for (int64_t k = 0; k < n; k++) {
        lbm_status st = benqueue_step(b, l, b->timing);
        if (st != LBM_OK) return st;
        if (b->timing && b->ev_used >= 8192) {
            st = bharvest(b);
            if (st != LBM_OK) return st;
        }
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(const lbm_config *configs, int32_t ncase, lbm_batch **out) {
    if (!configs || !out || ncase < 1) return bfail(nullptr, LBM_EINVAL, "bad batch arguments");
    *out = nullptr;
    for (int k = 0; k < ncase; k++)
        if (configs[k].collision != LBM_BGK || configs[k].boundary != LBM_HALFWAY)
            return bfail(nullptr, LBM_EINVAL,
                         "case %d: batches run BGK with the half-way boundary only", k);
    for (int k = 1; k < ncase; k++)
        if (configs[k].precision != configs[0].precision ||
            configs[k].rho_w_mode != configs[0].rho_w_mode ||
            configs[k].device != configs[0].device)
            return bfail(nullptr, LBM_EINVAL,
                         "case %d: precision, rho_w_mode and device must match case 0", k);
    if (cudaSetDevice(configs[0].device) != cudaSuccess)
        return bfail(nullptr, LBM_ECUDA, "cannot select device %d", configs[0].device);
    lbm_batch *b = new (std::nothrow) lbm_batch;
    if (!b) return bfail(nullptr, LBM_ENOMEM, "host allocation failed");
    b->device = configs[0].device;
    b->precision = configs[0].precision;
    b->rho_w_mode = configs[0].rho_w_mode;
    if (configs[0].stream) {
        b->stream = static_cast<cudaStream_t>(configs[0].stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            brelease(b);
            return bfail(nullptr, LBM_ECUDA, "stream creation failed");
        }
        b->own_stream = true;
    }
    b->cases.reserve(ncase);
    for (int k = 0; k < ncase; k++) {
        lbm_config g = configs[k];
        g.stream = b->stream;
        lbm_ctx *c = nullptr;
        lbm_status st = lbm_create(&g, &c);
        if (st != LBM_OK) {
            const std::string why = g_create_error;
            brelease(b);
            return bfail(nullptr, st, "case %d: %s", k, why.c_str());
        }
        c->batch = b;
        b->cases.push_back(c);
        if (g.body_force[0] != 0.0 || g.body_force[1] != 0.0) b->force = true;
    }
    const size_t n = (size_t)ncase;
    cudaError_t e = cudaMalloc(&b->cases_d, n * sizeof(StepParams));
    if (e == cudaSuccess) e = cudaMalloc(&b->counts_d, 3 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->active_d, n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->ticket_d, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&b->state_d, n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->drag_d, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b->calm_d, n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->anchor_d, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->calm_d, 0, n * sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaMalloc(&b->steps_d, n * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->toff_d, n * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->ioff_d, n * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&b->nactive_h, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->ticket_d, 0, sizeof(unsigned int), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->state_d, 0, n * sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->counts_d, 0, 3 * sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        brelease(b);
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA,
                     "lbm_batch_create: %s", cudaGetErrorString(e));
    }
    b->state.assign(n, LBM_CASE_ACTIVE);
    b->steps.assign(n, 0);
    b->drag.assign(n, std::nan(""));
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch *b) {
    if (!b) return LBM_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    brelease(b);
    return LBM_OK;
}

int32_t lbm_batch_size(const lbm_batch *b) { return b ? (int32_t)b->cases.size() : -1; }

lbm_status lbm_batch_case(lbm_batch *b, int32_t k, lbm_ctx **ctx) {
    if (!b || !ctx || k < 0 || k >= (int32_t)b->cases.size()) return LBM_EINVAL;
    *ctx = b->cases[k];
    return LBM_OK;
}

lbm_status lbm_batch_add_solid(lbm_batch *b, int32_t k, const lbm_disk *d, int32_t *id) {
    if (!b || !d || k < 0 || k >= (int32_t)b->cases.size()) return LBM_EINVAL;
    if (d->vx != 0.0 || d->vy != 0.0 || d->omega != 0.0 || d->motion != LBM_PRESCRIBED)
        return bfail(b, LBM_EINVAL, "solids of a batch rest (zero velocity, prescribed)");
    lbm_ctx *c = b->cases[k];
    BCK(b, cudaSetDevice(b->device));
    bdrop_graph(b);
    c->batch = nullptr;
    lbm_status st = lbm_add_solid(c, d, id);
    c->batch = b;
    if (st != LBM_OK) return bfail(b, st, "case %d: %s", k, c->err.c_str());
    b->dirty = true;
    return LBM_OK;
}

lbm_status lbm_batch_set_convergence(lbm_batch *b, int32_t every, double tol, int64_t max_steps) {
    if (!b || every < 1 || !(tol >= 0.0) || !std::isfinite(tol) || max_steps < 0)
        return LBM_EINVAL;
    b->every = every;
    b->tol = tol;
    b->max_steps = max_steps;
    b->dirty = true;
    bdrop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_set_convergence_window(lbm_batch *b, int32_t tests) {
    if (!b || tests < 1) return LBM_EINVAL;
    b->window = tests;
    b->dirty = true;
    bdrop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_run(lbm_batch *b, int64_t steps, int32_t *nactive) {
    if (!b || steps < 0) return LBM_EINVAL;
    BCK(b, cudaSetDevice(b->device));
    lbm_status st = bprepare(b);
    if (st != LBM_OK) return st;
    int64_t done = 0;
    int na = *b->nactive_h;
    while (done < steps && na > 0) {
        int64_t chunk = b->every - b->since_test;
        if (chunk > steps - done) chunk = steps - done;
        if (b->graph && !b->timing && chunk == b->every) {
            if (!b->gexec) {
                cudaGraph_t g;
                const int64_t before = b->launches;
                BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                st = bsteps(b, chunk);
                cudaError_t e = st == LBM_OK ? gbm::launch_batch_converge(
                                                   blaunch(b), bstate(b), gbm::BATCH_TEST, b->stream)
                                             : cudaSuccess;
                cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
                b->launches = before;  // counted when the graph is launched
                if (st != LBM_OK) return st;
                BCK(b, e);
                BCK(b, e2);
                e = cudaGraphInstantiate(&b->gexec, g, 0);
                cudaGraphDestroy(g);
                BCK(b, e);
            }
            BCK(b, cudaGraphLaunch(b->gexec, b->stream));
            b->launches += 2 * chunk + 1;
        } else {
            st = bsteps(b, chunk);
            if (st != LBM_OK) return st;
            if (b->since_test + chunk == b->every) {
                BCK(b, gbm::launch_batch_converge(blaunch(b), bstate(b), gbm::BATCH_TEST,
                                                  b->stream));
                b->launches++;
            }
        }
        done += chunk;
        b->since_test = (int)((b->since_test + chunk) % b->every);
        if (b->since_test == 0) {
            BCK(b, cudaMemcpyAsync(b->nactive_h, b->counts_d + 2, sizeof(int),
                                   cudaMemcpyDeviceToHost, b->stream));
            BCK(b, cudaStreamSynchronize(b->stream));
            na = *b->nactive_h;
        }
    }
    st = bharvest(b);
    if (st == LBM_OK) st = bgather(b);
    if (st != LBM_OK) return st;
    if (nactive) {
        int32_t a = 0;
        for (int32_t s : b->state) a += s == LBM_CASE_ACTIVE;
        *nactive = a;
    }
    return LBM_OK;
}

lbm_status lbm_batch_state(lbm_batch *b, int32_t *state, int64_t *steps, double *drag) {
    if (!b) return LBM_EINVAL;
    BCK(b, cudaSetDevice(b->device));
    lbm_status st = bgather(b);
    if (st != LBM_OK) return st;
    for (size_t k = 0; k < b->cases.size(); k++) {
        if (state) state[k] = b->state[k];
        if (steps) steps[k] = b->steps[k];
        if (drag) drag[k] = b->drag[k];
    }
    return LBM_OK;
}

lbm_status lbm_batch_retire(lbm_batch *b, const int32_t *ids, int32_t n) {
    if (!b || n < 0 || (n > 0 && !ids)) return LBM_EINVAL;
    BCK(b, cudaSetDevice(b->device));
    lbm_status st = bgather(b);
    if (st != LBM_OK) return st;
    for (int32_t i = 0; i < n; i++)
        if (ids[i] < 0 || ids[i] >= (int32_t)b->cases.size() || b->state[ids[i]] != LBM_CASE_ACTIVE)
            return bfail(b, LBM_EINVAL, "case %d is not active", ids[i]);
    const int32_t one = LBM_CASE_CONVERGED;
    for (int32_t i = 0; i < n; i++)
        BCK(b, cudaMemcpyAsync(b->state_d + ids[i], &one, sizeof one, cudaMemcpyHostToDevice,
                               b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    b->dirty = true;  // the lists are rebuilt before the next step
    st = bprepare(b);
    if (st == LBM_OK) st = bgather(b);
    return st;
}

lbm_status lbm_batch_set_launch(lbm_batch *b, int32_t variant, int32_t tile_rows,
                                int32_t persistent, int32_t graph) {
    if (!b || variant < 0 || variant > 2 || tile_rows < 1 || tile_rows > 64) return LBM_EINVAL;
    if (variant != b->variant || tile_rows != b->tile_h || (persistent != 0) != b->persistent)
        b->dirty = true;
    b->variant = variant;
    b->tile_h = tile_rows;
    b->persistent = persistent != 0;
    b->graph = graph != 0;
    bdrop_graph(b);
    return LBM_OK;
}

lbm_status lbm_batch_get_launch(const lbm_batch *b, int32_t *variant, int32_t *tile_rows,
                                int32_t *persistent) {
    if (!b) return LBM_EINVAL;
    if (variant) *variant = b->variant;
    if (tile_rows) *tile_rows = b->tile_h;
    if (persistent) *persistent = b->persistent ? 1 : 0;
    return LBM_OK;
}

lbm_status lbm_batch_set_timing(lbm_batch *b, int32_t enable) {
    if (!b) return LBM_EINVAL;
    BCK(b, cudaSetDevice(b->device));
    lbm_status st = bharvest(b);
    if (st != LBM_OK) return st;
    if (enable && !b->timing) {
        b->timed_ms = 0.0;
        b->timed_launches = 0;
    }
    b->timing = enable != 0;
    return LBM_OK;
}

lbm_status lbm_batch_get_timing(lbm_batch *b, double *ms, int64_t *launches) {
    if (!b) return LBM_EINVAL;
    BCK(b, cudaSetDevice(b->device));
    lbm_status st = bharvest(b);
    if (st != LBM_OK) return st;
    if (ms) *ms = b->timed_ms;
    if (launches) *launches = b->timed_launches;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int32_t steps, int32_t *best) {
    if (!b || steps < 1) return LBM_EINVAL;
    BCK(b, cudaSetDevice(b->device));
    lbm_status st = bharvest(b);
    if (st != LBM_OK) return st;
    const bool was_timing = b->timing;
    const double keep_ms = b->timed_ms;
    const int64_t keep_n = b->timed_launches;
    // {variant, rows per tile, persistent}
    static const int kShapes[][3] = {{0, 1, 0}, {1, 1, 0}, {2, 1, 0}, {0, 2, 0}, {1, 2, 0},
                                     {2, 2, 0}, {1, 4, 0}, {2, 4, 0}, {1, 1, 1}, {2, 1, 1}};
    double best_ms = 0.0;
    int pick = 0;
    const int nshape = (int)(sizeof kShapes / sizeof kShapes[0]);
    for (int k = 0; k < nshape; k++) {
        const int *sh = kShapes[k];
        if (sh[0] != b->variant || sh[1] != b->tile_h || (sh[2] != 0) != b->persistent)
            b->dirty = true;
        b->variant = sh[0];
        b->tile_h = sh[1];
        b->persistent = sh[2] != 0;
        st = bprepare(b);
        if (st != LBM_OK) return st;
        b->timing = true;
        st = bsteps(b, 1);  // the first launch of a kernel is not timed
        if (st == LBM_OK) st = bharvest(b);
        b->timed_ms = 0.0;
        b->timed_launches = 0;
        if (st == LBM_OK) st = bsteps(b, steps);
        if (st == LBM_OK) st = bharvest(b);
        if (st != LBM_OK) return st;
        const double ms = b->timed_ms / (b->timed_launches ? b->timed_launches : 1);
        if (k == 0 || ms < best_ms) {
            best_ms = ms;
            pick = k;
        }
    }
    b->dirty = true;
    b->variant = kShapes[pick][0];
    b->tile_h = kShapes[pick][1];
    b->persistent = kShapes[pick][2] != 0;
    b->timing = was_timing;
    b->timed_ms = keep_ms;
    b->timed_launches = keep_n;
    bdrop_graph(b);
    st = bprepare(b);  // rebuild for the chosen tiles; the drag history restarts
    if (st == LBM_OK) st = bgather(b);
    if (st != LBM_OK) return st;
    if (best) {
        best[0] = kShapes[pick][0];
        best[1] = kShapes[pick][1];
        best[2] = kShapes[pick][2];
    }
    return LBM_OK;
}

int64_t lbm_batch_launch_count(const lbm_batch *b) { return b ? b->launches : -1; }

const char *lbm_batch_last_error(const lbm_batch *b) {
    return b ? b->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
