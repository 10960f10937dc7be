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

using gbm::DSolid;
using gbm::StepParams;

struct lbm_ctx {
    lbm_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int pitch = 0;
    size_t elem = 0;
    void *f[2] = {nullptr, nullptr};
    uint16_t *owner = nullptr, *prev = nullptr, *flags = nullptr;
    DSolid *solids = nullptr;
    int solid_cap = 0;
    int nsolid = 0;
    int *moving_d = nullptr;
    int moving_cap = 0;
    std::vector<int> moving;
    std::vector<uint8_t> is_moving;
    double *ring = nullptr;
    int ring_cap = 0;      // solids the ring was laid out for
    long long *t_d = nullptr;
    int *status_d = nullptr;
    unsigned int *bar_d = nullptr;  // grid barrier of the per-solid kernel
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
    // staging buffer for host transfers
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
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
    p.prev = c->prev;
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
    p.precision = g.precision;
    p.sc_variant = c->sc_variant;
    p.omega_f = (float)(1.0 / g.tau);
    p.body_xf = (float)g.body_force[0];
    p.body_yf = (float)g.body_force[1];
    p.rho0_f = (float)g.rho0;
    p.bar = c->bar_d;
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
    void *bufs[] = {c->f[0], c->f[1], c->owner, c->prev, c->flags, c->solids, c->moving_d,
                    c->ring, c->t_d, c->status_d, c->bar_d, c->scratch};
    for (void *b : bufs)
        if (b) cudaFree(b);
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
    CK(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

// One step t -> t+1: the advection-collision kernel, then the per-solid work
// (link sums and force record of time t, motion, t += 1, re-rasterisation).
lbm_status enqueue_step(lbm_ctx *c, const StepParams &p, bool timed) {
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
    if (timed) {
        CK(c, cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
        c->ev_used += 2;
    }
    if (p.nsolid > 0) CK(c, gbm::launch_solids(p, p.nmoving > 0 ? gbm::SOLIDS_REMASK : 0, c->stream));
    else CK(c, gbm::launch_tick(p, c->stream));
    c->launches += 2;
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
    if (st & 1) return fail(c, LBM_EUNSTABLE, "non-finite or non-positive density produced");
    if (st & 2) return fail(c, LBM_EUNSTABLE, "a solid reached a non-finite state");
    if (st & 4) {
        // a grid barrier gave up: reset it so that later launches start clean
        cudaMemsetAsync(c->bar_d, 0, 2 * sizeof(unsigned int), c->stream);
        return fail(c, LBM_ETIMEOUT, "a grid-wide barrier of the per-solid kernel timed out");
    }
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
    if (g.reserved != 0) return fail(nullptr, LBM_EINVAL, "reserved must be 0");
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
    if (e == cudaSuccess) e = cudaMalloc(&c->owner, plane * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->prev, plane * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->flags, plane * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMalloc(&c->t_d, sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&c->status_d, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->bar_d, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->bar_d, 0, 2 * sizeof(unsigned int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->owner, 0xFF, plane * sizeof(uint16_t), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->prev, 0xFF, plane * sizeof(uint16_t), c->stream);
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
    cudaSetDevice(ctx->cfg.device);
    cudaStreamSynchronize(ctx->stream);
    release(ctx);
    return LBM_OK;
}

lbm_status lbm_add_solid(lbm_ctx *c, const lbm_disk *d, int32_t *id_out) {
    if (!c || !d) return LBM_EINVAL;
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
    s.pend_t = -1;
    s.near = 1;  // until the first pair test: assume a neighbour
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
                c->launches = before;  // counted when the graph is launched
                CK(c, cudaStreamEndCapture(c->stream, &graph));
                cudaError_t e = cudaGraphInstantiate(&c->gexec, graph, 0);
                cudaGraphDestroy(graph);
                CK(c, e);
            }
            CK(c, cudaGraphLaunch(c->gexec, c->stream));
            c->launches += 2 * (int64_t)c->graph_steps;
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
    for (int k = 0; k < 5; k++)
        if (!std::isfinite(state[k])) return fail(c, LBM_EINVAL, "non-finite solid state");
    CK(c, cudaSetDevice(c->cfg.device));
    DSolid s;
    CK(c, cudaMemcpyAsync(&s, c->solids + id, sizeof s, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (state[0] != s.x || state[1] != s.y)
        return fail(c, LBM_EINVAL, "lbm_set_solid changes velocities only; position must match");
    s.xa = s.xn = s.x;
    s.ya = s.yn = s.y;
    s.ta = c->t;
    s.vx = s.vxn = state[2];
    s.vy = s.vyn = state[3];
    s.om = s.omn = state[4];
    s.vxf = (float)state[2];
    s.vyf = (float)state[3];
    s.omf = (float)state[4];
    CK(c, cudaMemcpyAsync(c->solids + id, &s, sizeof s, cudaMemcpyHostToDevice, c->stream));
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
    if (!c || variant < 0 || variant > 2) return LBM_EINVAL;
    drop_graph(c);
    c->sc_variant = variant;
    return LBM_OK;
}

int32_t lbm_kernel_variant(const lbm_ctx *c) { return c ? c->sc_variant : -1; }

lbm_status lbm_autotune(lbm_ctx *c, int32_t steps, int32_t *best) {
    if (!c || steps < 1) return LBM_EINVAL;
    const bool was_timing = c->timing;
    const double keep_ms = c->timed_ms;
    const int64_t keep_n = c->timed_launches;
    lbm_status st = harvest_timing(c);
    if (st != LBM_OK) return st;
    double best_ms = 0.0;
    int best_v = 0;
    for (int v = 0; v <= 2; v++) {
        c->sc_variant = v;
        drop_graph(c);
        c->timing = true;
        c->timed_ms = 0.0;
        c->timed_launches = 0;
        st = lbm_step(c, 1);  // first launch of a variant is not timed
        if (st == LBM_OK) st = harvest_timing(c);
        c->timed_ms = 0.0;
        c->timed_launches = 0;
        if (st == LBM_OK) st = lbm_step(c, steps);
        if (st == LBM_OK) st = harvest_timing(c);
        if (st != LBM_OK) return st;
        const double ms = c->timed_ms / (c->timed_launches ? c->timed_launches : 1);
        if (v == 0 || ms < best_ms) {
            best_ms = ms;
            best_v = v;
        }
    }
    c->sc_variant = best_v;
    c->timing = was_timing;
    c->timed_ms = keep_ms;
    c->timed_launches = keep_n;
    if (best) *best = best_v;
    return LBM_OK;
}

}  // extern "C"
