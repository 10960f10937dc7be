"""Learned warm start of steady channel flows past fixed disks.

Host-side orchestration only: every step runs in the library's kernels (the
batch engine for the lattice-Boltzmann runs, the U-Net kernels for training
and inference, ``lbm_warm_start`` for the initial state).  PyTorch supplies
device buffers.  The library's contexts and the network run on streams of
their own: every hand-over of device data between them and PyTorch's stream
waits for the producer (torch.cuda.synchronize).

  steady(cases)          run a batch of cases to a steady state (drag change
                         below tol per `every` steps) and collect the fields
                         and each case's network input (lbm_case_input: the
                         solid mask, Re and geometric features)
  dataset(cases, runs)   network inputs, targets (scaled residuals of rho
                         and u) and fluid masks
  train(net, data, ...)  mini-batch Adam on the masked MSE
  time_to_drag(...)      steps and wall time until every case's drag is within
                         rel of its converged value, from the plain (cold)
                         initial state or from the network's prediction (warm),
                         with the drift check and the fallback to a cold start

Targets are residuals from the empty channel's Poiseuille flow (u_P(y) the
inlet parabola, rho_P(x) its linear pressure drop; lbm_warm_start adds them
back), scaled per case (U = peak inlet speed): u - u_P = U p_u,
rho - rho_P = (100 U^2 / Re) p_rho, so that both are of order one from Re = 1
to 100 and vanish away from the disks.
"""

from __future__ import annotations

import time

import numpy as np

from . import lbm as L


# The reference of the time-to-drag measurement: the plain run until its drag
# has stayed within REF_TOL (relative) of one value for REF_WINDOW tests 100
# steps apart, at most REF_CAP steps.  A single test of the change over 100
# steps passes at a turning point of an oscillating drag, and in FP32 the
# drag's round-off noise is a few 1e-7 per 100 steps (a band of about 5e-6
# over 10^4 steps); a band of 1e-5 held for 5000 steps is above that noise and
# leaves the drag within REF_TOL * T / 5000 of the steady value for an
# approach of decay time T (T is at most about 1.5e4 steps on these channels).
REF_TOL = 1e-5
REF_WINDOW = 50
REF_CAP = 600_000


def poiseuille(case):
    """(rho_P [ny][nx], u_P [ny]) of the case's empty channel."""
    nx, ny = case["nx"], case["ny"]
    h = float(ny)
    yy = np.arange(ny) + 0.5
    nu = (case["tau"] - 0.5) / 3.0
    u = 4.0 * case["inflow_umax"] * yy * (h - yy) / (h * h)
    rho = case.get("rho0", 1.0) + 24.0 * nu * case["inflow_umax"] * (nx - 1 - np.arange(nx)) / (h * h)
    return np.broadcast_to(rho[None, :], (ny, nx)), u


def rho_scale(case) -> float:
    return 100.0 * case["u_scale"] ** 2 / case["re"]


def _batch(cases, precision, device, stream, ring=4):
    return L.Batch.from_workloads(cases, precision=precision, force_ring=ring, device=device,
                                  stream=stream)


def inputs(b, cases, device=0):
    """Network inputs [N][8][ny][nx] (device tensor) of the cases of batch b."""
    import torch

    ny, nx = cases[0]["ny"], cases[0]["nx"]
    x = torch.empty((len(cases), 8, ny, nx), dtype=torch.float32,
                    device=torch.device("cuda", device))
    torch.cuda.synchronize(device)  # x is allocated on PyTorch's stream
    for k in range(len(cases)):
        L.lbm_case_input(b.case(k).handle, cases[k]["re"], x[k])
    torch.cuda.synchronize(device)  # written on the batch's stream
    return x


def steady(cases, *, precision=L.LBM_FP32_DEV, tol=1e-7, every=100, cap=300_000, chunk=1000,
           window=1, device=0, stream=None, fields=True):
    """Run every case to a steady state (drag change below tol per `every`
    steps in `window` consecutive tests); returns dict with state, steps,
    drag and (with fields) rho, ux, uy [N][ny][nx] (NaN at solids) and the
    network inputs x [N][8][ny][nx]."""
    b = _batch(cases, precision, device, stream)
    xin = inputs(b, cases, device).cpu().numpy() if fields else None
    b.set_convergence(every=every, tol=tol, max_steps=cap, window=window)
    t0 = time.perf_counter()
    while b.run(chunk) > 0:
        pass
    wall = time.perf_counter() - t0
    st, steps, drag = b.state()
    out = dict(state=st, steps=steps, drag=drag, wall=wall)
    if fields:
        ny, nx = cases[0]["ny"], cases[0]["nx"]
        rho = np.empty((len(cases), ny, nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        for k in range(len(cases)):
            if st[k] == L.LBM_CASE_UNSTABLE:  # no usable state to read
                rho[k] = ux[k] = uy[k] = np.nan
            else:
                rho[k], ux[k], uy[k] = b.case(k).fields()
        out.update(rho=rho, ux=ux, uy=uy, x=xin)
    b.close()
    return out


def dataset(cases, runs, mirror=False, rho_weight=1.0):
    """Inputs [N][8][H][W], targets [N][3][H][W], fluid [N][H][W] (float32) of
    the cases that reached a steady state; with mirror, each also mirrored
    about the channel's centre line (y -> ny - 1 - y, u_y -> -u_y, and the
    input's antisymmetric coordinate plane negated), which the walls and the
    inlet profile leave invariant.  The density target is multiplied by
    rho_weight (its weight in the squared-error loss is rho_weight^2;
    time_to_drag divides it out again)."""
    keep = np.flatnonzero(runs["state"] == L.LBM_CASE_CONVERGED)
    n = len(keep)
    ny, nx = cases[0]["ny"], cases[0]["nx"]
    x = np.ascontiguousarray(runs["x"][keep], dtype=np.float32)
    y = np.zeros((n, 3, ny, nx), dtype=np.float32)
    f = np.zeros((n, ny, nx), dtype=np.float32)
    for j, k in enumerate(keep):
        solid = np.isnan(runs["rho"][k])
        U = cases[k]["u_scale"]
        f[j] = ~solid
        rp, up = poiseuille(cases[k])
        y[j, 0] = np.where(solid, 0.0, (runs["rho"][k] - rp) * rho_weight / rho_scale(cases[k]))
        y[j, 1] = np.where(solid, 0.0, (runs["ux"][k] - up[:, None]) / U)
        y[j, 2] = np.where(solid, 0.0, runs["uy"][k] / U)
    if mirror:
        xm, ym, fm = x[:, :, ::-1].copy(), y[:, :, ::-1].copy(), f[:, ::-1].copy()
        xm[:, 7] *= -1.0
        ym[:, 2] *= -1.0
        x, y, f = np.concatenate([x, xm]), np.concatenate([y, ym]), np.concatenate([f, fm])
    return dict(x=x, y=y, fluid=f, index=keep)


def train(net, data, *, epochs=20, batch=16, lr=1e-3, lr_end=1e-4, seed=0, log=None):
    """Mini-batch Adam over the dataset (held on the device); the learning
    rate decays geometrically from lr to lr_end.  Returns the epoch losses."""
    import torch

    dev = torch.device("cuda", net.cfg.device)
    X = torch.from_numpy(data["x"]).to(dev)
    Y = torch.from_numpy(data["y"]).to(dev)
    F = torch.from_numpy(data["fluid"]).to(dev)
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    steps = max(1, epochs * (n // batch))
    k = 0
    for ep in range(epochs):
        order = rng.permutation(n)
        tot, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = torch.from_numpy(order[s:s + batch]).to(dev)
            xb, yb, fb = X[idx].contiguous(), Y[idx].contiguous(), F[idx].contiguous()
            torch.cuda.current_stream(dev).synchronize()  # gathered on PyTorch's stream
            rate = lr * (lr_end / lr) ** (k / steps)
            tot += L.lbm_unet_train_step(net.handle, xb, yb, fb, batch, rate, on_device=True)
            cnt += 1
            k += 1
        losses.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep} loss {losses[-1]:.4e}")
    return losses


def predict(net, data_x, batch=16):
    """Network outputs for inputs [N][8][H][W] (host), as a device tensor."""
    import torch

    dev = torch.device("cuda", net.cfg.device)
    X = torch.from_numpy(data_x).to(dev)
    out = torch.empty((X.shape[0], 3, X.shape[2], X.shape[3]), dtype=torch.float32, device=dev)
    chunks = [X[s:min(X.shape[0], s + batch)].contiguous() for s in range(0, X.shape[0], batch)]
    torch.cuda.synchronize(dev)  # uploaded on PyTorch's stream
    for k, xc in enumerate(chunks):
        s = k * batch
        L.lbm_unet_forward(net.handle, xc, out[s:s + xc.shape[0]], xc.shape[0], on_device=True)
    torch.cuda.synchronize(dev)  # written on the network's stream
    return out


def band_step(anchor, calm, drag, tol):
    """One test of the steady band: a case whose drag is within tol
    (relative) of its anchor counts one more calm test; any other case starts
    a new run at its current drag.  Returns the new (anchor, calm) arrays;
    NaN anchors start a run."""
    near = np.abs(drag - anchor) < tol * np.abs(drag)
    return np.where(near, anchor, drag), np.where(near, calm + 1, 0)


def _mass(ctx):
    """Total fluid mass of a case, or NaN once its state is unusable."""
    try:
        return float(np.nansum(ctx.fields()[0]))
    except L.LBMError:
        return float("nan")


def time_to_drag(cases, d_star, *, net=None, rel=1e-4, precision=L.LBM_FP32_DEV, every=100,
                 cap=300_000, drift_steps=200, drift_mass=1e-2, settle=REF_TOL,
                 settle_checks=REF_WINDOW, flux=True, rho_weight=1.0, device=0, stream=None):
    """Steps and wall time until every case's Eq. 5 drag is within rel of
    d_star (the converged drag of the plain run), starting cold (net None)
    or warm from the network's prediction (on the channel's Poiseuille flow,
    with each column's mass flux made equal to the inlet's unless flux is
    False: lbm_warm_start; the network's density channel in units of
    rho_scale / rho_weight).  The plain run is the judge, and
    a warm case falls back to it: its populations are reset to the plain
    initial state in place (it keeps stepping in the batch, its count of
    steps goes on):
      - after drift_steps, when its state is unstable, its drag not finite or
        its total mass has moved by more than drift_mass (relative);
      - whenever its drag has settled away from d_star (stayed within settle,
        relative, of one value for settle_checks blocks of `every` steps in
        a row, the reference's own steady test): it has reached another
        steady state.
    A case stops stepping once it is within rel of d_star.  The wall time
    covers input assembly, inference and every step."""
    import torch

    dev = torch.device("cuda", device)
    b = _batch(cases, precision, device, stream)
    b.set_convergence(every=every, tol=0.0, max_steps=cap)  # retire only at the cap
    n = len(cases)
    ny, nx = cases[0]["ny"], cases[0]["nx"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fallback = np.zeros(n, dtype=bool)
    elsewhere = np.zeros(n, dtype=bool)
    mass0 = None
    if net is not None:
        # the plain initial state of every case, for the cold restarts
        f_cold = torch.empty((n, 9, ny, nx), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        for k in range(n):
            L.lbm_get_populations(b.case(k).handle, f_cold[k], on_device=True)
        xin = inputs(b, cases, device)
        out = torch.empty((n, 3, ny, nx), dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        for s in range(0, n, net.max_batch):
            e = min(n, s + net.max_batch)
            L.lbm_unet_forward(net.handle, xin[s:e], out[s:e], e - s, on_device=True)
        torch.cuda.synchronize()
        for k in range(n):
            L.lbm_warm_start(b.case(k).handle, out[k], cases[k]["u_scale"],
                             rho_scale(cases[k]) / rho_weight, base=True, flux=flux)
        mass0 = np.array([_mass(b.case(k)) for k in range(n)])
    done = np.full(n, -1, dtype=np.int64)
    drift = None
    anchor = np.full(n, np.nan)  # drag at the start of the current calm run
    calm = np.zeros(n, dtype=np.int64)  # blocks in a row within settle of the anchor
    steps = 0

    def restart_cold(ids):
        for k in ids:
            L.lbm_set_populations(b.case(k).handle, f_cold[k], on_device=True)
        torch.cuda.synchronize()
        fallback[ids] = True
        calm[ids] = 0
        anchor[ids] = np.nan

    while steps < cap:
        b.run(every)
        steps += every
        st, stp, drag = b.state()
        active = (done < 0) & (st == L.LBM_CASE_ACTIVE)
        if net is not None and steps == drift_steps:
            drift = np.zeros(n)
            bad = []
            for k in range(n):
                m = _mass(b.case(k))
                drift[k] = abs(m - mass0[k]) / abs(mass0[k]) if np.isfinite(m) else np.inf
                if st[k] == L.LBM_CASE_UNSTABLE or not np.isfinite(drag[k]) or \
                        not drift[k] <= drift_mass:
                    bad.append(k)
            bad = np.array(bad, dtype=np.int64)
            if len(bad):
                unstable = bad[st[bad] == L.LBM_CASE_UNSTABLE]
                if len(unstable):  # retired by the batch: its plain run, in a batch of its own
                    r = time_to_drag([cases[k] for k in unstable], d_star[unstable], rel=rel,
                                     precision=precision, every=every, cap=cap, device=device,
                                     stream=stream)
                    done[unstable] = np.where(r["steps"] >= 0, r["steps"] + steps, -1)
                    fallback[unstable] = True
                restart_cold(bad[st[bad] == L.LBM_CASE_ACTIVE])
                continue  # the restarted cases' drag is not yet meaningful
        ok = np.abs(drag - d_star) <= rel * np.abs(d_star)
        newly = ok & active
        done[newly] = steps
        if newly.any():  # the case has reached its drag: it stops stepping
            b.retire(np.flatnonzero(newly))
        if net is not None and steps > drift_steps:
            anchor, calm = band_step(anchor, calm, drag, settle)
            away = (calm >= settle_checks) & ~ok & active & ~fallback
            if away.any():
                elsewhere |= away
                restart_cold(np.flatnonzero(away))
        if (done >= 0).all():
            break
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    b.close()
    return dict(steps=done, wall=wall, fallback=fallback, elsewhere=elsewhere, batch_steps=steps,
                drift=drift if net is not None and steps >= drift_steps else None)
